// Persistent tile-queue step over a batch of resident shots (FP32 in increment form, one block per
// shot).
//
// One launch advances every active shot of the batch by one leapfrog step.  Its CTAs (a fixed
// number per SM) pull work items from one device-wide queue -- an interior tile of a shot (128
// columns x `rows` rows of the column-marching stencil) or a boundary-strip tile of a shot
// (closures, SAT terms, strip point sources) -- until the queue is empty; the items of a step are
// independent (they read level n and write level n+1 of disjoint nodes).  The last CTA to finish
// (detected with a fence and a counter, no waiting) adds the point-source nodes off the strips,
// advances each active shot (parity, time, steps left) and resets the queue for the next launch.
// A CUDA graph of K such launches is the batch's K-step loop; shots are admitted and retired by
// the host between graph launches.
#pragma once
#include "sbp_interior_march.cuh"
#include "sbp_kernels.cuh"

namespace sbp {

// immutable description of a resident shot
struct alignas(64) BatchShot {
    MarchMaps maps;                 // tensor maps of the shot's u[0], u[1], c (global memory: 64-byte aligned)
    BlockDev view;
    const int4* tiles;              // the shot's strip tiles (k_strip_tile numbering, with source ranges)
    const SrcNode* ssrc;            // strip point-source nodes (by tile) or null
    const SrcNode* isrc;            // point-source nodes off the strips or null
    const SrcParam* spar;
    int nisrc;
    int rows;                       // rows of an interior item
    double dt, dt2, beta;
    float dt2f;
};

// mutable per-shot state, advanced by the last CTA of every launch
struct BatchState {
    int remaining;                  // steps left (0: nothing to do)
    int cur;                        // index of the current level in BlockDev::u
    double t;                       // time of the current level
};

struct BatchHead {
    const int4* items;              // (shot, kind 0 interior / 1 strip, item index, 0)
    int nitems;
    int nshots;
    const BatchShot* shots;
    BatchState* state;
    int next;                       // queue position (reset by the last CTA)
    int done;                       // CTAs finished (reset by the last CTA)
};

template <int O> constexpr size_t batch_smem_bytes() {
    return MarchCfg<O>::BYTES > StripTile<O>::template bytes<float>() ? MarchCfg<O>::BYTES
                                                                        : StripTile<O>::template bytes<float>();
}

template <int O>
__global__ void __launch_bounds__(MTHREADS, 4) k_batch_step(BatchHead* __restrict__ H, int* err) {
    extern __shared__ __align__(128) unsigned char batch_smem[];
    // the item's step arguments and (interior items) the block fields the march reads, kept in
    // shared memory for the item: the launch-per-step kernels read them from the constant bank,
    // here they would otherwise be re-read from global memory inside the row loop
    __shared__ StepArgs s_a;
    __shared__ MarchView s_v;
    __shared__ int4 s_w;
    __shared__ int s_item, s_run;
    __shared__ int s_last;
    const int tx = threadIdx.x;
    for (;;) {
        if (tx == 0) {
            const int it = atomicAdd(&H->next, 1);
            int run = 0;
            if (it < H->nitems) {
                const int4 w = H->items[it];
                const BatchState st = H->state[w.x];
                if (st.remaining > 0) {
                    run = 1;
                    const BatchShot& sh = H->shots[w.x];
                    StepArgs a{};
                    a.cur = st.cur;
                    a.with_data = 1;
                    a.t = st.t;
                    a.dt = sh.dt;
                    a.dt2 = sh.dt2;
                    a.dt2f = sh.dt2f;
                    s_a = a;
                    if (w.y == 0) s_v = march_view(sh.view);
                }
                s_w = w;
            }
            s_item = it;
            s_run = run;
        }
        __syncthreads();
        const int it = s_item, run = s_run;
        const int4 w = s_w;
        __syncthreads();                                    // s_item, s_run, s_w are rewritten only after every thread read them
        if (it >= H->nitems) break;
        if (!run) continue;
        const BatchShot& sh = H->shots[w.x];
        bool ok;
        if (w.y == 0) ok = march_tile<O, 3>(sh.maps, s_v, s_a, sh.rows, w.z, err, batch_smem);
        else ok = strip_tile_body<float, O, 0, MTHREADS>(&sh.view, sh.tiles[w.z], s_a, sh.beta, err, sh.ssrc, sh.spar,
                                                        batch_smem);
        __syncthreads();                                    // the next item reuses the shared memory
        if (!ok) break;                                     // uniform: set by a CTA-wide vote
    }
    // retirement: the last CTA sees every other CTA's stores (each fenced before its count)
    __threadfence();
    __syncthreads();
    if (tx == 0) s_last = atomicAdd(&H->done, 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int s = 0; s < H->nshots; ++s) {
        const BatchState st = H->state[s];
        if (st.remaining <= 0) continue;
        const BatchShot& sh = H->shots[s];
        StepArgs a{};
        a.t = st.t;
        const size_t plane = (size_t)sh.view.n2 * sh.view.pitch;
        float* Un = reinterpret_cast<float*>(sh.view.u[1 - st.cur]);
        float* DU = reinterpret_cast<float*>(sh.view.du);
        const float* Wv = reinterpret_cast<const float*>(sh.view.w);
        for (int k = tx; k < sh.nisrc; k += blockDim.x) {     // as k_sources (leapfrog mode)
            const SrcNode nd = sh.isrc[k];
            const double Wt = ricker_at(sh.spar[nd.src], a);
            const double fac = sh.dt2 * (double)Wv[nd.gi] * Wt;
            atomicAdd(Un + nd.gi, float(fac * nd.wt0));
            atomicAdd(Un + plane + nd.gi, float(fac * nd.wt1));
            atomicAdd(DU + nd.gi, float(fac * nd.wt0));
            atomicAdd(DU + plane + nd.gi, float(fac * nd.wt1));
        }
    }
    __syncthreads();
    for (int s = tx; s < H->nshots; s += blockDim.x) {
        BatchState& st = H->state[s];
        if (st.remaining <= 0) continue;
        st.remaining -= 1;
        st.cur = 1 - st.cur;
        st.t += H->shots[s].dt;
    }
    if (tx == 0) {
        H->next = 0;
        H->done = 0;
    }
}

}  // namespace sbp
