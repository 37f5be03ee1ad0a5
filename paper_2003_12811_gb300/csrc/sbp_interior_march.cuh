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
//  * 1/(rho J) and u^{n-1} of the output row are loaded from global memory two rows ahead.
#pragma once
#include <cuda.h>
#include "sbp_device.cuh"
#include "sbp_interior_tma.cuh"

namespace sbp {

constexpr int MTHREADS = 128, MBOXW = 140, MXOFF = 8, MR = 2, MNCH = 4;

template <int O> struct MarchCfg {
    static constexpr int Q = Ord<O>::Q;
    // ring slot: displacement box [2][MR][W] padded to a 128-byte multiple, then the
    // coefficient box [10][MR][W]; the slot itself is padded to 128 bytes (TMA destinations)
    static constexpr int UPAD = ((2 * MR * MBOXW * 4 + 127) / 128) * 128 / 4;
    static constexpr int CHUNK = ((UPAD + 10 * MR * MBOXW) * 4 + 127) / 128 * 128 / 4;
    static constexpr int G1 = 2 * 2 * MBOXW;                 // [row parity][component][col]
    static constexpr size_t BYTES = (size_t)(MNCH * CHUNK + G1) * 4 + 64;
};

struct MarchMaps {
    CUtensorMap u[2];   // [2][n2][pitch], box [2][MR][MBOXW]
    CUtensorMap c;      // [10][n2][pitch], box [10][MR][MBOXW]
};

// tile geometry shared with the host: first column, columns per CTA, rows per CTA
__host__ __device__ inline int march_x0(int strip) { return (strip / 4) * 4; }

template <int O, int MODE>
__global__ void __launch_bounds__(MTHREADS, 4)
k_interior_march(const __grid_constant__ MarchMaps maps, BlockDev B, StepArgs a, int rows_per_cta, int* err) {
    using MC = MarchCfg<O>;
    constexpr int Q = MC::Q, W = MBOXW, L = 2 * Q + 1;
    extern __shared__ __align__(128) unsigned char march_smem[];
    float* ring = reinterpret_cast<float*>(march_smem);
    float* g1s = ring + MNCH * MC::CHUNK;
    uint64_t* bars = reinterpret_cast<uint64_t*>(g1s + MC::G1);

    const int S = B.strip, n1 = B.n1, n2 = B.n2, P = B.pitch;
    const int lim1 = n1 - S, lim2 = n2 - S;
    const int X0 = march_x0(S);
    const int ncx = (lim1 - X0 + MTHREADS - 1) / MTHREADS;
    const int cx = blockIdx.x % ncx, cy = blockIdx.x / ncx;
    const int x0 = X0 + cx * MTHREADS;
    const int ys = S + cy * rows_per_cta;
    if (ys >= lim2) return;
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
    auto rowp = [&](int r) -> const float* {
        const int rr = r - rb;
        return ring + ((rr / MR) % MNCH) * MC::CHUNK + (rr % MR) * W;
    };
    auto poff = [](int p) { return p < 2 ? p * MR * W : MC::UPAD + (p - 2) * MR * W; };
    auto at = [&](int p, int r, int col) -> float { return rowp(r)[poff(p) + col]; };
    auto wait_row = [&](int r) -> bool {        // called when row r is the first row of a chunk
        const int ch = (r - rb) / MR;
        return mbar_wait_bounded(&bars[ch % MNCH], (ch / MNCH) & 1);
    };

    float ak[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) ak[k] = Ord<O>::template aT<float>(k);
    const float ih1 = B.ih1f, ih2 = B.ih2f;
    const float ih11 = ih1 * ih1, ih22 = ih2 * ih2;

    // register queues, index 0 = oldest row (qb: rows r-q+1 .. r+q of the c_2j2l fields)
    constexpr int LB = 2 * Q;
    float qu0[L], qu1[L], qb0[LB], qb1[LB], qb2[LB], qg0[L], qg1[L], qh0[L], qh1[L];
#pragma unroll
    for (int k = 0; k < L; ++k) qu0[k] = qu1[k] = qg0[k] = qg1[k] = qh0[k] = qh1[k] = 0.f;
#pragma unroll
    for (int k = 0; k < LB; ++k) qb0[k] = qb1[k] = qb2[k] = 0.f;
    // delay lines of the y edge fluxes: fy*[m-1][0] = F_m(r-m) .. fy*[m-1][m-1] = F_m(r-1)
    float fy0[Q][Q], fy1[Q][Q];
#pragma unroll
    for (int m = 0; m < Q; ++m)
#pragma unroll
        for (int k = 0; k < Q; ++k) fy0[m][k] = fy1[m][k] = 0.f;
    // threads 0..2Q-1 also follow one halo column each (x0-Q..x0-1, x0+128..x0+127+Q) for g1
    const int hc = tx < Q ? MXOFF - Q + tx : MXOFF + MTHREADS + (tx - Q);
    const bool halo = tx < 2 * Q;
    // prefetched 1/(rho J) and u^{n-1}: *_c for the row being output, *_n for the next row
    float w_c = 0.f, u0_c = 0.f, u1_c = 0.f, w_n = 0.f, u0_n = 0.f, u1_n = 0.f;
    auto load_row = [&](int r, float& wv, float& v0, float& v1) {
        if (MODE == 0 && col_ok && r >= ys && r < ye) {
            const size_t gi = (size_t)r * P + gx;
            wv = __ldg(reinterpret_cast<const float*>(B.w) + gi);
            const float* Un = reinterpret_cast<const float*>(B.u[1 - a.cur]);
            v0 = Un[gi];
            v1 = Un[gi + plane];
        }
    };
    load_row(ys, w_c, u0_c, u1_c);
    load_row(ys + 1, w_n, u0_n, u1_n);
    auto rotate = [&](int r) {   // after row r: current <- next, next <- row r + 2
        w_c = w_n;
        u0_c = u0_n;
        u1_c = u1_n;
        load_row(r + 2, w_n, u0_n, u1_n);
    };

    bool ok = true;
    int waited = 0;                               // chunks whose completion every thread has seen
    int next_issue = MNCH < nchunks ? MNCH : nchunks;   // meaningful in thread 0 only
    // the march: step r consumes lookahead row Lr = r + Q; outputs row r when r >= ys
    for (int r = rb - Q; r < ye; ++r) {
        const int Lr = r + Q;
        if (((Lr - rb) % MR) == 0) {
            ok = wait_row(Lr) && ok;
            ++waited;
        }
        // --- lookahead row: own-column values into the queues, g2 at (x, Lr)
        {
            const float* pL = rowp(Lr) + cc;
            const float u0n = pL[poff(0)], u1n = pL[poff(1)];
            float d0 = 0.f, d1 = 0.f;
#pragma unroll
            for (int k = 1; k <= Q; ++k) {
                d0 += ak[k - 1] * (pL[poff(0) + k] - pL[poff(0) - k]);
                d1 += ak[k - 1] * (pL[poff(1) + k] - pL[poff(1) - k]);
            }
            d0 *= ih1;
            d1 *= ih1;
            const float m6 = pL[poff(8)], m7 = pL[poff(9)], m8 = pL[poff(10)], m9 = pL[poff(11)];
#pragma unroll
            for (int k = 0; k < L - 1; ++k) {
                qu0[k] = qu0[k + 1]; qu1[k] = qu1[k + 1];
                qg0[k] = qg0[k + 1]; qg1[k] = qg1[k + 1];
            }
#pragma unroll
            for (int k = 0; k < LB - 1; ++k) {
                qb0[k] = qb0[k + 1]; qb1[k] = qb1[k + 1]; qb2[k] = qb2[k + 1];
            }
            qu0[L - 1] = u0n;
            qu1[L - 1] = u1n;
            qb0[LB - 1] = pL[poff(5)];
            qb1[LB - 1] = pL[poff(6)];
            qb2[LB - 1] = pL[poff(7)];
            qg0[L - 1] = m6 * d0 + m8 * d1;       // g2_1 = c_1121 D_1 u_1 + c_1221 D_1 u_2
            qg1[L - 1] = m7 * d0 + m9 * d1;       // g2_2 = c_1122 D_1 u_1 + c_1222 D_1 u_2
            if (halo) {
#pragma unroll
                for (int k = 0; k < L - 1; ++k) {
                    qh0[k] = qh0[k + 1];
                    qh1[k] = qh1[k + 1];
                }
                qh0[L - 1] = at(0, Lr, hc);
                qh1[L - 1] = at(1, Lr, hc);
            }
        }
        // --- narrow y in edge-flux form: F_m(r) from the queued rows, F_m(r-m) from the delay
        // lines (needed from the first output row on, so formed from row ys - Q on)
        float ry0 = 0.f, ry1 = 0.f;
        if (r >= ys - Q) {
            const float uc0 = qu0[Q], uc1 = qu1[Q];
#pragma unroll
            for (int m = 1; m <= Q; ++m) {
                auto B0p = [&](int k) { return qb0[k + Q - 1]; };
                auto B1p = [&](int k) { return qb1[k + Q - 1]; };
                auto B2p = [&](int k) { return qb2[k + Q - 1]; };
                const float e0 = Edge<O>::template e<float>(m, B0p), e1 = Edge<O>::template e<float>(m, B1p),
                            e2 = Edge<O>::template e<float>(m, B2p);
                const float dp0 = qu0[Q + m] - uc0, dp1 = qu1[Q + m] - uc1;
                const float f0 = e0 * dp0 + e1 * dp1, f1 = e1 * dp0 + e2 * dp1;
                ry0 += f0 - fy0[m - 1][0];
                ry1 += f1 - fy1[m - 1][0];
#pragma unroll
                for (int k = 0; k < m - 1; ++k) {
                    fy0[m - 1][k] = fy0[m - 1][k + 1];
                    fy1[m - 1][k] = fy1[m - 1][k + 1];
                }
                fy0[m - 1][m - 1] = f0;
                fy1[m - 1][m - 1] = f1;
            }
        }
        if (r < ys) continue;                    // queue fill (prologue)
        // --- g1 at (x, r) into the shared row
        const int par = r & 1;
        {
            float d0 = 0.f, d1 = 0.f;
#pragma unroll
            for (int k = 1; k <= Q; ++k) {
                d0 += ak[k - 1] * (qu0[Q + k] - qu0[Q - k]);
                d1 += ak[k - 1] * (qu1[Q + k] - qu1[Q - k]);
            }
            d0 *= ih2;
            d1 *= ih2;
            const float* pr0 = rowp(r) + cc;
            const float m6 = pr0[poff(8)], m7 = pr0[poff(9)], m8 = pr0[poff(10)], m9 = pr0[poff(11)];
            g1s[(par * 2 + 0) * W + cc] = m6 * d0 + m7 * d1;
            g1s[(par * 2 + 1) * W + cc] = m8 * d0 + m9 * d1;
        }
        // halo columns of g1 (x0-Q .. x0-1 and x0+128 .. x0+127+Q), from the halo queues
        if (halo) {
            float d0 = 0.f, d1 = 0.f;
#pragma unroll
            for (int k = 1; k <= Q; ++k) {
                d0 += ak[k - 1] * (qh0[Q + k] - qh0[Q - k]);
                d1 += ak[k - 1] * (qh1[Q + k] - qh1[Q - k]);
            }
            d0 *= ih2;
            d1 *= ih2;
            const float m6 = at(8, r, hc), m7 = at(9, r, hc), m8 = at(10, r, hc), m9 = at(11, r, hc);
            g1s[(par * 2 + 0) * W + hc] = m6 * d0 + m7 * d1;
            g1s[(par * 2 + 1) * W + hc] = m8 * d0 + m9 * d1;
        }
        if (__syncthreads_or(!ok)) {
            // a bounded wait ran out: record it, drain this CTA's issued copies (bounded), stop
            if (tx == 0) {
                atomicOr(err, 4);
                for (int ch = waited; ch < next_issue; ++ch) mbar_wait_bounded(&bars[ch % MNCH], (ch / MNCH) & 1);
            }
            __syncthreads();
            return;
        }
        // every thread is past row r-1: ring slots holding only rows below r can be refilled
        if (tx == 0) {
            const int below = (r - rb) / MR;      // chunks entirely below row r
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
        const float uc0 = pr[poff(0)], uc1 = pr[poff(1)];
        float rx0 = 0.f, rx1 = 0.f;
#pragma unroll
        for (int m = 1; m <= Q; ++m) {
            auto B0p = [&](int k) { return pr[poff(2) + k]; };
            auto B1p = [&](int k) { return pr[poff(3) + k]; };
            auto B2p = [&](int k) { return pr[poff(4) + k]; };
            auto B0m = [&](int k) { return pr[poff(2) - m + k]; };
            auto B1m = [&](int k) { return pr[poff(3) - m + k]; };
            auto B2m = [&](int k) { return pr[poff(4) - m + k]; };
            const float e0p = Edge<O>::template e<float>(m, B0p), e1p = Edge<O>::template e<float>(m, B1p),
                        e2p = Edge<O>::template e<float>(m, B2p);
            const float e0m = Edge<O>::template e<float>(m, B0m), e1m = Edge<O>::template e<float>(m, B1m),
                        e2m = Edge<O>::template e<float>(m, B2m);
            const float dp0 = pr[poff(0) + m] - uc0, dp1 = pr[poff(1) + m] - uc1;
            const float dm0 = pr[poff(0) - m] - uc0, dm1 = pr[poff(1) - m] - uc1;
            rx0 += e0p * dp0 + e1p * dp1 + e0m * dm0 + e1m * dm1;
            rx1 += e1p * dp0 + e2p * dp1 + e1m * dm0 + e2m * dm1;
        }
        float r0 = rx0 * ih11 + ry0 * ih22;
        float r1 = rx1 * ih11 + ry1 * ih22;
        // --- mixed: D_1 g1 from the shared row, D_2 g2 from the queue
        float m10 = 0.f, m11 = 0.f, m20 = 0.f, m21 = 0.f;
        const float* g10 = g1s + (par * 2 + 0) * W + cc;
        const float* g11 = g1s + (par * 2 + 1) * W + cc;
#pragma unroll
        for (int k = 1; k <= Q; ++k) {
            m10 += ak[k - 1] * (g10[k] - g10[-k]);
            m11 += ak[k - 1] * (g11[k] - g11[-k]);
            m20 += ak[k - 1] * (qg0[Q + k] - qg0[Q - k]);
            m21 += ak[k - 1] * (qg1[Q + k] - qg1[Q - k]);
        }
        r0 += m10 * ih1 + m20 * ih2;
        r1 += m11 * ih1 + m21 * ih2;
        const size_t gi = (size_t)r * P + gx;
        if (a.with_data && B.jf) {
            const float* __restrict__ JF = reinterpret_cast<const float*>(B.jf);
            #pragma unroll
                for (int kb = 0; kb < 8; ++kb) {
                    if (kb >= a.K) break;
                r0 += (float)a.Tk[kb] * JF[(size_t)kb * plane + gi];
                r1 += (float)a.Tk[kb] * JF[(size_t)(a.K + kb) * plane + gi];
            }
        }
        if (MODE == 0) {
            float* __restrict__ Un = reinterpret_cast<float*>(B.u[1 - a.cur]);
            const float dt2 = a.dt2f;
            Un[gi] = 2.f * uc0 - u0_c + dt2 * w_c * r0;
            Un[gi + plane] = 2.f * uc1 - u1_c + dt2 * w_c * r1;
        } else {
            float* __restrict__ R = reinterpret_cast<float*>(B.r);
            R[gi] = r0;
            R[gi + plane] = r1;
        }
        rotate(r);
    }
    // every issued chunk has been waited for inside the march (the last lookahead rows cover
    // the last chunk), so no bulk copy is still in flight when the CTA exits
}

}  // namespace sbp
