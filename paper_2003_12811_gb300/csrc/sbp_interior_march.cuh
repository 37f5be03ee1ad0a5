// FP32 interior stencil, column-marching form (sm_103a).
//
// Same arithmetic as k_interior (Sec. 4.6; narrow rows through edge weights, mixed terms
// D_1 (c_1j2l D_2 u_l) + D_2 (c_2j1l D_1 u_l)), laid out so that shared memory carries only
// the x-neighbour traffic:
//  * a CTA of 128 threads owns 128 adjacent interior columns and a band of rows; thread x
//    marches down its column;
//  * rows stream through a ring of NCH chunks of R rows in shared memory, each chunk filled by
//    two cp.async.bulk.tensor.3d boxes (displacement [2][R][140], coefficients [10][R][140],
//    x from the tile start - 8) tracked by an mbarrier per ring slot (bounded waits);
//  * the y-direction stencils use register queues of the thread's own column (displacement and
//    the fluxes g2 = c_1l2j D_1 u_l for the last 2q+1 rows, the three c_2j2l fields for rows
//    r-q+1..r+q); the narrow y rows are written in edge-flux form
//      h^2 D_yy(b) u |_r = sum_m F_m(r) - F_m(r-m),  F_m(r) = E_m(r) (u_{r+m} - u_r),
//    so every edge weight E_m is formed once and F_m waits m rows in a short delay line;
//  * the x-direction fluxes g1 = c_1j2l D_2 u_l of the current row are exchanged through a
//    double-buffered shared row (one barrier per row);
//  * 1/(rho J) and u^{n-1} of the output row are loaded from global memory two rows ahead;
//  * MODE 0: leapfrog update from the two levels; 3: leapfrog update in increment form (the
//    FP32 state: d^{n+1} = d^n + dt^2 w r, u^{n+1} = u^n + d^{n+1}, see leapfrog_store);
//    1: operator output r; 2: RK4 stage (rk4_store);
//  * the two components of the displacement and of every flux are carried as float2 and
//    combined with packed FP32x2 instructions (one issue slot for both).
#pragma once
#include <cuda.h>
#include <type_traits>
#include "sbp_device.cuh"

namespace sbp {

constexpr int MTHREADS = 128, MBOXW = 140, MXOFF = 8, MR = 2, MNCH = 4;

template <int O> struct MarchCfg {
    static constexpr int Q = Ord<O>::Q;
    // ring slot: displacement box [2][MR][W] padded to a 128-byte multiple, then the
    // coefficient box [10][MR][W]; the slot itself is padded to 128 bytes (TMA destinations)
    static constexpr int UPAD = ((2 * MR * MBOXW * 4 + 127) / 128) * 128 / 4;
    static constexpr int CHUNK = ((UPAD + 10 * MR * MBOXW) * 4 + 127) / 128 * 128 / 4;
    static constexpr int G1 = 2 * 2 * MBOXW;                 // [row parity][col][component] (float2)
    static constexpr int HQ = 6 * 8 * 2;                      // halo queues [2q][8] (float2), persistent callers
    static constexpr size_t BYTES = (size_t)(MNCH * CHUNK + G1 + HQ) * 4 + 64;
};

struct MarchMaps {
    CUtensorMap u[2];   // [2][n2][pitch], box [2][MR][MBOXW]
    CUtensorMap c;      // [10][n2][pitch], box [10][MR][MBOXW]
};

// packed FP32x2 arithmetic (one instruction for both halves)
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// interior edge weight E_m of one field as an explicit FMA chain in a fixed order: every copy of
// the row loop (prologue, unrolled output rows) rounds it the same way, so the result at a node
// does not depend on how the rows are split between CTAs
template <int O, class F> __device__ __forceinline__ float edge1(int m, F B) {
    float acc = 0.f;
#pragma unroll
    for (int k = EdgeRange<O>::LO; k <= EdgeRange<O>::HI; ++k) {
        const float c = edge_w<O>(m, k);
        if (c != 0.f) acc = __fmaf_rn(c, B(k), acc);
    }
    return acc;
}

// tile geometry shared with the host: first column, columns per CTA, rows per CTA
__host__ __device__ inline int march_x0(int strip) { return (strip / 4) * 4; }

// columns-of-128 tiles across the interior of a block (the host sizes grids and work lists with it)
__host__ __device__ inline int march_ncx(int n1, int strip) { return (n1 - strip - march_x0(strip) + MTHREADS - 1) / MTHREADS; }

// The block fields the tile reads, as a compact copy (a persistent caller keeps it in shared memory;
// the launch-per-step kernels read the BlockDev kernel parameter directly).
struct MarchView {
    int n1, n2, pitch, strip;
    float ih1f, ih2f;
    void* u[2];
    void* du;
    const void* w;
    const void* jf;
    void* r;
};
__host__ __device__ inline MarchView march_view(const BlockDev& B) {
    MarchView v;
    v.n1 = B.n1;
    v.n2 = B.n2;
    v.pitch = B.pitch;
    v.strip = B.strip;
    v.ih1f = B.ih1f;
    v.ih2f = B.ih2f;
    v.u[0] = B.u[0];
    v.u[1] = B.u[1];
    v.du = B.du;
    v.w = B.w;
    v.jf = B.jf;
    v.r = B.r;
    return v;
}

// One interior tile: the 128 columns of column tile `tile % ncx` and the rows_per_cta rows of row
// band `tile / ncx`, by the 128 threads of the calling CTA, with `smem` (MarchCfg<O>::BYTES, 128-byte
// aligned) as its ring, flux row and mbarriers.  Returns false when a bounded wait ran out (the
// error word is set; the tile's copies have been drained).  The mbarriers are invalidated before
// the return, so a persistent caller can reuse the shared memory for its next tile after a
// CTA barrier.
template <int O, int MODE, class BV = BlockDev>
__device__ __forceinline__ bool march_tile(const MarchMaps& maps, const BV& B, const StepArgs& a, int rows_per_cta,
                                           int tile, int* err, unsigned char* march_smem) {
    using MC = MarchCfg<O>;
    constexpr int Q = MC::Q, W = MBOXW, L = 2 * Q + 1;
    float* ring = reinterpret_cast<float*>(march_smem);
    float* g1s = ring + MNCH * MC::CHUNK;
    float2* hqs = reinterpret_cast<float2*>(g1s + MC::G1);
    uint64_t* bars = reinterpret_cast<uint64_t*>(g1s + MC::G1 + MC::HQ);
    // a persistent caller (view type other than the BlockDev kernel parameter) keeps the halo
    // columns' displacement queues in shared memory (rows indexed mod 8) instead of registers:
    // its block fields live in registers, not in the constant bank
    constexpr bool HS = !std::is_same<BV, BlockDev>::value;

    const int S = B.strip, n1 = B.n1, n2 = B.n2, P = B.pitch;
    const int lim1 = n1 - S, lim2 = n2 - S;
    const int X0 = march_x0(S);
    const int ncx = march_ncx(n1, S);
    const int cx = tile % ncx, cy = tile / ncx;
    const int x0 = X0 + cx * MTHREADS;
    const int ys = S + cy * rows_per_cta;
    if (ys >= lim2) return true;
    const int ye = min(lim2, ys + rows_per_cta);
    const int rb = ys - Q;                       // first row streamed into the ring
    const int tx = threadIdx.x;
    const int gx = x0 + tx;
    const bool col_ok = gx >= S && gx < lim1;
    const int cc = tx + MXOFF;                   // column of this thread inside a ring row
    const size_t plane = (size_t)n2 * P;
    const CUtensorMap* umap = &maps.u[a.cur];
    const CUtensorMap* cmap = &maps.c;
    constexpr uint32_t BYTES_U = 2 * MR * W * 4, BYTES_C = 10 * MR * W * 4;
    const int nrows = ye + Q - rb;               // rows streamed
    const int nchunks = (nrows + MR - 1) / MR;

    if (tx == 0) {
        for (int k = 0; k < MNCH; ++k) mbar_init(&bars[k], 1);
        fence_barrier_init();
        fence_proxy_async();
    }
    __syncthreads();
    auto issue = [&](int ch) {
        float* dst = ring + (ch % MNCH) * MC::CHUNK;
        uint64_t* bar = &bars[ch % MNCH];
        mbar_expect_tx(bar, BYTES_U + BYTES_C);
        tma_load_3d(dst, umap, x0 - MXOFF, rb + ch * MR, 0, bar);
        tma_load_3d(dst + MC::UPAD, cmap, x0 - MXOFF, rb + ch * MR, 0, bar);
    };
    if (tx == 0)
        for (int ch = 0; ch < MNCH && ch < nchunks; ++ch) issue(ch);

    // ring access: rowp(r) points at (plane 0, row r, column 0) of row r's slot; plane p
    // (0,1 displacement; 2..11 coefficient planes 0..9) is at the compile-time offset poff(p)
    auto rowp = [&](int r) -> const float* {     // r >= rb: unsigned division is a shift
        const unsigned rr = (unsigned)(r - rb);
        return ring + ((rr / MR) % MNCH) * MC::CHUNK + (rr % MR) * W;
    };
    auto poff = [](int p) { return p < 2 ? p * MR * W : MC::UPAD + (p - 2) * MR * W; };
    auto at = [&](int p, int r, int col) -> float { return rowp(r)[poff(p) + col]; };
    auto wait_row = [&](int r) -> bool {        // called when row r is the first row of a chunk
        const unsigned ch = (unsigned)(r - rb) / MR;
        return mbar_wait_bounded(&bars[ch % MNCH], (ch / MNCH) & 1);
    };

    float ak[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) ak[k] = Ord<O>::template aT<float>(k);
    const float ih1 = B.ih1f, ih2 = B.ih2f;
    const float ih11 = ih1 * ih1, ih22 = ih2 * ih2;

    // the two displacement components (and the two components of every flux) travel together
    // as float2 and are combined with packed FP32x2 arithmetic.  Register queues, index 0 =
    // oldest row: qu displacement, qg fluxes g2, qh halo displacement (rows r-q..r+q); qb the
    // c_2j2l fields (c_2121, c_2122) and qc (c_2222) for rows r-q+1..r+q
    constexpr int LB = 2 * Q;
    float2 qu[L], qg[L], qh[L], qb[LB];
    float qc[LB];
#pragma unroll
    for (int k = 0; k < L; ++k) qu[k] = qg[k] = qh[k] = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < LB; ++k) {
        qb[k] = make_float2(0.f, 0.f);
        qc[k] = 0.f;
    }
    // delay lines of the y edge fluxes: fy[m-1][0] = F_m(r-m) .. fy[m-1][m-1] = F_m(r-1)
    float2 fy[Q][Q];
#pragma unroll
    for (int m = 0; m < Q; ++m)
#pragma unroll
        for (int k = 0; k < Q; ++k) fy[m][k] = make_float2(0.f, 0.f);
    // threads 0..2Q-1 also follow one halo column each (x0-Q..x0-1, x0+128..x0+127+Q) for g1
    const int hc = tx < Q ? MXOFF - Q + tx : MXOFF + MTHREADS + (tx - Q);
    const bool halo = tx < 2 * Q;
    // prefetched 1/(rho J) and u^{n-1} (MODE 3: the increment d^n): *_c for the row being output,
    // *_n for the next row
    float w_c = 0.f, w_n = 0.f;
    float2 up_c = make_float2(0.f, 0.f), up_n = make_float2(0.f, 0.f);
    auto load_row = [&](int r, float& wv, float2& v) {
        if (MODE != 1 && col_ok && r >= ys && r < ye) {
            const size_t gi = (size_t)r * P + gx;
            wv = __ldg(reinterpret_cast<const float*>(B.w) + gi);
            if (MODE == 0 || MODE == 3) {
                const float* Up = reinterpret_cast<const float*>(MODE == 3 ? B.du : B.u[1 - a.cur]);
                v = make_float2(Up[gi], Up[gi + plane]);
            }
        }
    };
    load_row(ys, w_c, up_c);
    load_row(ys + 1, w_n, up_n);
    auto rotate = [&](int r) {   // after row r: current <- next, next <- row r + 2
        w_c = w_n;
        up_c = up_n;
        load_row(r + 2, w_n, up_n);
    };
    // displacement pair / field pairs at ring offset o of a row pointer
    auto U2 = [&](const float* p, int o) { return make_float2(p[poff(0) + o], p[poff(1) + o]); };
    auto X2 = [&](const float* p, int o) { return make_float2(p[poff(2) + o], p[poff(3) + o]); };

    bool ok = true;
    int waited = 0;                               // chunks whose completion every thread has seen
    int next_issue = MNCH < nchunks ? MNCH : nchunks;   // meaningful in thread 0 only
    // the march: step r consumes lookahead row Lr = r + Q and outputs row r when r >= ys.
    // look(r) pushes row Lr into the queues; yflux() forms the y edge fluxes of the queue centre
    auto look = [&](int r) {
        const int Lr = r + Q;
        if (((unsigned)(Lr - rb) % MR) == 0) {
            ok = wait_row(Lr) && ok;
            ++waited;
        }
        // --- lookahead row: own-column values into the queues, g2 at (x, Lr)
        {
            const float* pL = rowp(Lr) + cc;
            float2 d = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 1; k <= Q; ++k) d = ffma2(bc2(ak[k - 1]), fsub2(U2(pL, k), U2(pL, -k)), d);
            d = fmul2(d, bc2(ih1));
            const float m6 = pL[poff(8)], m7 = pL[poff(9)], m8 = pL[poff(10)], m9 = pL[poff(11)];
#pragma unroll
            for (int k = 0; k < L - 1; ++k) {
                qu[k] = qu[k + 1];
                qg[k] = qg[k + 1];
            }
#pragma unroll
            for (int k = 0; k < LB - 1; ++k) {
                qb[k] = qb[k + 1];
                qc[k] = qc[k + 1];
            }
            qu[L - 1] = U2(pL, 0);
            qb[LB - 1] = make_float2(pL[poff(5)], pL[poff(6)]);
            qc[LB - 1] = pL[poff(7)];
            // g2_1 = c_1121 D_1 u_1 + c_1221 D_1 u_2,  g2_2 = c_1122 D_1 u_1 + c_1222 D_1 u_2
            qg[L - 1] = ffma2(make_float2(m6, m7), bc2(d.x), fmul2(make_float2(m8, m9), bc2(d.y)));
            if (halo) {
                if constexpr (HS) {
                    hqs[tx * 8 + ((unsigned)Lr & 7u)] = make_float2(at(0, Lr, hc), at(1, Lr, hc));
                } else {
#pragma unroll
                    for (int k = 0; k < L - 1; ++k) qh[k] = qh[k + 1];
                    qh[L - 1] = make_float2(at(0, Lr, hc), at(1, Lr, hc));
                }
            }
        }
    };
    auto yflux = [&]() -> float2 {
        // --- narrow y in edge-flux form: F_m(r) from the queued rows, F_m(r-m) from the delay
        // lines (needed from the first output row on, so formed from row ys - Q on)
        float2 ry = make_float2(0.f, 0.f);
        {
#pragma unroll
            for (int m = 1; m <= Q; ++m) {
                float2 e01 = make_float2(0.f, 0.f);
#pragma unroll
                for (int k = EdgeRange<O>::LO; k <= EdgeRange<O>::HI; ++k) {
                    const float c = edge_w<O>(m, k);
                    if (c != 0.f) e01 = ffma2(bc2(c), qb[k + Q - 1], e01);
                }
                const float e2 = edge1<O>(m, [&](int k) { return qc[k + Q - 1]; });
                const float2 dp = fsub2(qu[Q + m], qu[Q]);
                // (F0, F1) = (e0, e1) dp_1 + (e1, e2) dp_2
                const float2 f = ffma2(e01, bc2(dp.x), fmul2(make_float2(e01.y, e2), bc2(dp.y)));
                ry = fadd2(ry, fsub2(f, fy[m - 1][0]));
#pragma unroll
                for (int k = 0; k < m - 1; ++k) fy[m - 1][k] = fy[m - 1][k + 1];
                fy[m - 1][m - 1] = f;
            }
        }
        return ry;
    };
    // prologue: fill the queues, then the delay lines; the output rows follow in a loop of its
    // own, unrolled so that the queue shifts become register renames
    for (int r = rb - Q; r < ys - Q; ++r) look(r);
    for (int r = ys - Q; r < ys; ++r) {
        look(r);
        (void)yflux();
    }
#pragma unroll 4
    for (int r = ys; r < ye; ++r) {
        look(r);
        const float2 ry = yflux();
        // --- g1 at (x, r) into the shared row
        const int par = r & 1;
        {
            float2 d = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 1; k <= Q; ++k) d = ffma2(bc2(ak[k - 1]), fsub2(qu[Q + k], qu[Q - k]), d);
            d = fmul2(d, bc2(ih2));
            const float* pr0 = rowp(r) + cc;
            const float m6 = pr0[poff(8)], m7 = pr0[poff(9)], m8 = pr0[poff(10)], m9 = pr0[poff(11)];
            // g1_1 = c_1121 D_2 u_1 + c_1122 D_2 u_2,  g1_2 = c_1221 D_2 u_1 + c_1222 D_2 u_2
            const float2 g = ffma2(make_float2(m6, m8), bc2(d.x), fmul2(make_float2(m7, m9), bc2(d.y)));
            reinterpret_cast<float2*>(g1s)[par * W + cc] = g;
        }
        // halo columns of g1 (x0-Q .. x0-1 and x0+128 .. x0+127+Q), from the halo queues
        if (halo) {
            float2 d = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 1; k <= Q; ++k) {
                if constexpr (HS)
                    d = ffma2(bc2(ak[k - 1]), fsub2(hqs[tx * 8 + ((unsigned)(r + k) & 7u)], hqs[tx * 8 + ((unsigned)(r - k) & 7u)]), d);
                else
                    d = ffma2(bc2(ak[k - 1]), fsub2(qh[Q + k], qh[Q - k]), d);
            }
            d = fmul2(d, bc2(ih2));
            const float m6 = at(8, r, hc), m7 = at(9, r, hc), m8 = at(10, r, hc), m9 = at(11, r, hc);
            const float2 g = ffma2(make_float2(m6, m8), bc2(d.x), fmul2(make_float2(m7, m9), bc2(d.y)));
            reinterpret_cast<float2*>(g1s)[par * W + hc] = g;
        }
        if (__syncthreads_or(!ok)) {
            // a bounded wait ran out: record it, drain this CTA's issued copies (bounded), stop
            if (tx == 0) {
                atomicOr(err, ERR_MARCH_WAIT);
                for (int ch = waited; ch < next_issue; ++ch) mbar_wait_bounded(&bars[ch % MNCH], (ch / MNCH) & 1);
            }
            __syncthreads();
            return false;
        }
        // every thread is past row r-1: ring slots holding only rows below r can be refilled
        if (tx == 0) {
            const int below = (int)((unsigned)(r - rb) / MR);   // chunks entirely below row r
            bool fenced = false;
            while (next_issue < nchunks && next_issue < below + MNCH) {
                if (!fenced) {
                    fence_proxy_async();
                    fenced = true;
                }
                issue(next_issue++);
            }
        }
        if (!col_ok) { rotate(r); continue; }
        // --- narrow x: edge weights from the x fields of row r (columns x-Q-2 .. x+Q)
        const float* pr = rowp(r) + cc;
        const float2 uc = qu[Q];                  // row r of this column (queue centre)
        float2 rx = make_float2(0.f, 0.f);
#pragma unroll
        for (int m = 1; m <= Q; ++m) {
            float2 e01p = make_float2(0.f, 0.f), e01m = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = EdgeRange<O>::LO; k <= EdgeRange<O>::HI; ++k) {
                const float c = edge_w<O>(m, k);
                if (c != 0.f) {
                    e01p = ffma2(bc2(c), X2(pr, k), e01p);
                    e01m = ffma2(bc2(c), X2(pr, k - m), e01m);
                }
            }
            const float e2p = edge1<O>(m, [&](int k) { return pr[poff(4) + k]; });
            const float e2m = edge1<O>(m, [&](int k) { return pr[poff(4) - m + k]; });
            const float2 dp = fsub2(U2(pr, m), uc), dm = fsub2(U2(pr, -m), uc);
            rx = ffma2(e01p, bc2(dp.x), rx);
            rx = ffma2(make_float2(e01p.y, e2p), bc2(dp.y), rx);
            rx = ffma2(e01m, bc2(dm.x), rx);
            rx = ffma2(make_float2(e01m.y, e2m), bc2(dm.y), rx);
        }
        float2 rr = ffma2(rx, bc2(ih11), fmul2(ry, bc2(ih22)));
        // --- mixed: D_1 g1 from the shared row, D_2 g2 from the queue
        float2 m1 = make_float2(0.f, 0.f), m2 = make_float2(0.f, 0.f);
        const float2* g1r = reinterpret_cast<const float2*>(g1s) + par * W + cc;
#pragma unroll
        for (int k = 1; k <= Q; ++k) {
            m1 = ffma2(bc2(ak[k - 1]), fsub2(g1r[k], g1r[-k]), m1);
            m2 = ffma2(bc2(ak[k - 1]), fsub2(qg[Q + k], qg[Q - k]), m2);
        }
        rr = ffma2(m1, bc2(ih1), rr);
        rr = ffma2(m2, bc2(ih2), rr);
        float r0 = rr.x, r1 = rr.y;
        const size_t gi = (size_t)r * P + gx;
        if (a.with_data && B.jf) {
            const float* __restrict__ JF = reinterpret_cast<const float*>(B.jf);
#pragma unroll
            for (int kb = 0; kb < 8; ++kb) {
                if (kb >= a.K) break;
                r0 = __fmaf_rn((float)a.Tk[kb], JF[(size_t)kb * plane + gi], r0);
                r1 = __fmaf_rn((float)a.Tk[kb], JF[(size_t)(a.K + kb) * plane + gi], r1);
            }
        }
        if (MODE == 0) {
            float* __restrict__ Un = reinterpret_cast<float*>(B.u[1 - a.cur]);
            const float2 nu = ffma2(bc2(a.dt2f * w_c), make_float2(r0, r1), fsub2(fadd2(uc, uc), up_c));
            Un[gi] = nu.x;
            Un[gi + plane] = nu.y;
        } else if (MODE == 3) {
            float* __restrict__ Un = reinterpret_cast<float*>(B.u[1 - a.cur]);
            float* __restrict__ DU = reinterpret_cast<float*>(B.du);
            const float2 d = ffma2(bc2(a.dt2f * w_c), make_float2(r0, r1), up_c);
            const float2 nu = fadd2(uc, d);
            Un[gi] = nu.x;
            Un[gi + plane] = nu.y;
            DU[gi] = d.x;
            DU[gi + plane] = d.y;
        } else if constexpr (MODE == 2) {
            rk4_store<float>(B, a, gi, plane, w_c, r0, r1);
        } else {
            float* __restrict__ R = reinterpret_cast<float*>(B.r);
            R[gi] = r0;
            R[gi + plane] = r1;
        }
        rotate(r);
    }
    // every issued chunk has been waited for inside the march (the last lookahead rows cover
    // the last chunk), so no bulk copy is still in flight when the CTA exits; the barriers are
    // invalidated once every thread is past its last wait
    __syncthreads();
    if (tx == 0)
        for (int k = 0; k < MNCH; ++k) mbar_inval(&bars[k]);
    return true;
}

template <int O, int MODE>
__global__ void __launch_bounds__(MTHREADS, 4)
k_interior_march(const __grid_constant__ MarchMaps maps, BlockDev B, StepArgs a, int rows_per_cta, int* err) {
    extern __shared__ __align__(128) unsigned char march_smem[];
    (void)march_tile<O, MODE>(maps, B, a, rows_per_cta, blockIdx.x, err, march_smem);
}

// The interior tiles of several blocks in one launch: CTA k takes tile k - start[b] of the block b
// with start[b] <= k < start[b + 1], so the CTAs of the next block fill the tail of the previous
// one instead of waiting for a launch boundary.
constexpr int MARCH_MAX_BLOCKS = 8;
struct MarchMulti {
    MarchMaps maps[MARCH_MAX_BLOCKS];
    BlockDev b[MARCH_MAX_BLOCKS];
    int start[MARCH_MAX_BLOCKS + 1];
    int rows[MARCH_MAX_BLOCKS];
    int nb;
};

template <int O, int MODE>
__global__ void __launch_bounds__(MTHREADS, 4)
k_interior_march_multi(const __grid_constant__ MarchMulti mm, StepArgs a, int* err) {
    extern __shared__ __align__(128) unsigned char march_smem[];
    const int k = blockIdx.x;
    int b = 0;
    while (b + 1 < mm.nb && k >= mm.start[b + 1]) ++b;
    (void)march_tile<O, MODE>(mm.maps[b], mm.b[b], a, mm.rows[b], k - mm.start[b], err, march_smem);
}

}  // namespace sbp
