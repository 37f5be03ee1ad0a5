// FP32 interior stencil with TMA-staged tiles (sm_103a).
//
// Same arithmetic as k_interior (Sec. 4.6: narrow rows through edge weights, mixed terms
// D_1 (c_1j2l D_2 u_l) + D_2 (c_2j1l D_1 u_l)), organised for HBM streaming:
//  * persistent CTAs walk the tiles of the interior region (tile = 32 x 16 output nodes);
//  * one elected thread issues cp.async.bulk.tensor.3d loads of the tile plus halo for the
//    10 coefficient planes (one box [10][TY+2Q][40]) and the 2 displacement planes
//    ([2][TY+2Q][40]); completion is tracked by mbarriers (transaction bytes);
//  * as soon as the edge weights and mixed fluxes of a tile are in shared memory, the loads
//    of the next tile are issued, so they overlap the output phase of the current tile;
//  * every mbarrier wait is bounded: on timeout the kernel records an error flag, drains
//    its own copies (bounded) and returns.
// The box starts 4 columns left of the tile (16-byte aligned x coordinate, as TMA requires);
// tiles start at column tile_x0(strip) + 32 k (the box may start at x = -4, which TMA fills with
// zeros); nodes outside the interior region are masked.
#pragma once
#include <cuda.h>
#include "sbp_device.cuh"

namespace sbp {

constexpr int TTX = 32, TTY = 16, TTHREADS = 256, TBOXW = 40, TXOFF = 4;
// first tile column: the largest multiple of 4 not above the strip width (16-byte aligned box start)
__host__ __device__ constexpr int tile_x0(int strip) { return (strip / 4) * 4; }

template <int O> struct TmaTile {
    static constexpr int Q = Ord<O>::Q;
    static constexpr int SY = TTY + 2 * Q;             // rows in a loaded box
    static constexpr int SX = TTX + 2 * Q;             // columns used by the mixed fluxes g1
    static constexpr int EX = TTX + Q, EY = TTY + Q;
    static constexpr int CBUF = 10 * SY * TBOXW;
    static constexpr int UBUF = 2 * SY * TBOXW;
    static constexpr int G1 = 2 * TTY * SX, G2 = 2 * SY * TTX;
    static constexpr int EXN = 9 * TTY * EX, EYN = 9 * EY * TTX;
    static constexpr int FLOATS = CBUF + 2 * UBUF + G1 + G2 + EXN + EYN;
    static constexpr size_t BYTES = (size_t)FLOATS * 4 + 128;   // + mbarriers
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: returns false after ~2^22 unsuccessful polls
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    for (int i = 0; i < (1 << 22); ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_barrier_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

struct TmaMaps {
    CUtensorMap u[2];   // displacement buffers: [2][n2][pitch], box [2][SY][40]
    CUtensorMap c;      // coefficients: [10][n2][pitch], box [10][SY][40]
};

template <int O, int MODE>
__global__ void __launch_bounds__(TTHREADS, 2)
k_interior_tma(const __grid_constant__ TmaMaps maps, BlockDev B, StepArgs a, int* err) {
    using TT = TmaTile<O>;
    constexpr int Q = TT::Q, SY = TT::SY, SX = TT::SX, EX = TT::EX, EY = TT::EY, W = TBOXW;
    extern __shared__ __align__(128) unsigned char tma_smem[];
    float* cbuf = reinterpret_cast<float*>(tma_smem);     // [10][SY][W]
    float* ubuf = cbuf + TT::CBUF;                         // [2 stages][2][SY][W]
    float* sg1 = ubuf + 2 * TT::UBUF;                      // [2][TY][SX]   col index c + Q
    float* sg2 = sg1 + TT::G1;                             // [2][SY][TX]
    float* sex = sg2 + TT::G2;                             // [3][Q][TY][EX] col index i + Q
    float* sey = sex + TT::EXN;                            // [3][Q][EY][TX] row index j + Q
    uint64_t* bars = reinterpret_cast<uint64_t*>(sey + TT::EYN);   // [0] c, [1],[2] u stages

    const int S = B.strip;
    const int n1 = B.n1, n2 = B.n2, P = B.pitch;
    const int lim1 = n1 - S, lim2 = n2 - S;
    const int TX0 = tile_x0(S);
    const int ntx = (lim1 - TX0 + TTX - 1) / TTX;
    const int nty = (lim2 - S + TTY - 1) / TTY;
    const int ntiles = ntx * nty;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const size_t plane = (size_t)n2 * P;
    const CUtensorMap* umap = &maps.u[a.cur];
    const CUtensorMap* cmap = &maps.c;
    constexpr uint32_t CBYTES = TT::CBUF * 4, UBYTES = TT::UBUF * 4;

    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init(&bars[2], 1);
        fence_barrier_init();
        fence_proxy_async();
    }
    __syncthreads();

    auto tile_origin = [&](int t, int& x0, int& y0) {
        const int by = t / ntx;
        x0 = TX0 + (t - by * ntx) * TTX;
        y0 = S + by * TTY;
    };
    auto issue = [&](int t, int stage, bool with_c) {
        int x0, y0;
        tile_origin(t, x0, y0);
        if (with_c) {
            mbar_expect_tx(&bars[0], CBYTES);
            tma_load_3d(cbuf, cmap, x0 - TXOFF, y0 - Q, 0, &bars[0]);
        }
        mbar_expect_tx(&bars[1 + stage], UBYTES);
        tma_load_3d(ubuf + stage * TT::UBUF, umap, x0 - TXOFF, y0 - Q, 0, &bars[1 + stage]);
    };

    int tile = blockIdx.x;
    if (tile >= ntiles) return;
    if (threadIdx.x == 0) issue(tile, 0, true);

    const float ih1 = B.ih1f, ih2 = B.ih2f;
    const float ih11 = ih1 * ih1, ih22 = ih2 * ih2;
    float ak[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) ak[k] = Ord<O>::template aT<float>(k);

    for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
        const int s = it & 1;
        bool ok = mbar_wait_bounded(&bars[0], it & 1) && mbar_wait_bounded(&bars[1 + s], (it >> 1) & 1);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicOr(err, 2);
                // drain this CTA's own copies (bounded) before the shared memory is released
                mbar_wait_bounded(&bars[0], it & 1);
                mbar_wait_bounded(&bars[1 + s], (it >> 1) & 1);
            }
            __syncthreads();
            return;
        }
        int x0, y0;
        tile_origin(tile, x0, y0);
        const float* su = ubuf + s * TT::UBUF;
        // early global loads of this thread's 1/(rho J) and u^{n-1} (two adjacent rows): they
        // complete while phase 2 runs
        const int pr0 = 2 * ty;                       // phase-3 rows pr0, pr0 + 1
        const int gx = x0 + tx;
        float wv[2] = {0.f, 0.f}, up0[2] = {0.f, 0.f}, up1[2] = {0.f, 0.f};
        bool act[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int gy = y0 + pr0 + k;
            act[k] = gx >= S && gx < lim1 && gy < lim2;
            if (MODE == 0 && act[k]) {
                const size_t gi = (size_t)gy * P + gx;
                wv[k] = __ldg(reinterpret_cast<const float*>(B.w) + gi);
                const float* Un = reinterpret_cast<const float*>(B.u[1 - a.cur]);
                up0[k] = Un[gi];
                up1[k] = Un[gi + plane];
            }
        }
        // ---- phase 2: mixed fluxes and edge weights, as warp-uniform tasks of 32 lanes:
        //   [0,16)      g1 = c_1j2l D_2 u_l, tile row t, tile columns
        //   [16,19)     g1 at the 2Q halo columns (96 lanes: row, halo column)
        //   [19,19+SY)  g2 = c_1l2j D_1 u_l, rows [-Q, TY+Q), tile columns
        //   next 16     x edge weights, tile row, i in [0, TX)
        //   next 2      x edge weights at i in [-Q, 0) (16 x Q lanes)
        //   next EY     y edge weights, j in [-Q, TY), tile columns
        constexpr int T_G1 = 0, T_G1H = TTY, T_G2 = T_G1H + (TTY * 2 * Q + 31) / 32, T_EX = T_G2 + SY,
                      T_EXH = T_EX + TTY, T_EY = T_EXH + (TTY * Q + 31) / 32, T_END = T_EY + EY;
        auto g1_at = [&](int r, int c) {           // c: column index in [0, SX) (tile column c - Q)
            const int col = c - Q + TXOFF;
            const float* p0 = su + (r + Q) * W + col;
            const float* p1 = p0 + SY * W;
            float d0 = 0.f, d1 = 0.f;
#pragma unroll
            for (int k = 1; k <= Q; ++k) {
                d0 += ak[k - 1] * (p0[k * W] - p0[-k * W]);
                d1 += ak[k - 1] * (p1[k * W] - p1[-k * W]);
            }
            d0 *= ih2;
            d1 *= ih2;
            const int mi = (r + Q) * W + col;
            const float m6 = cbuf[6 * SY * W + mi], m7 = cbuf[7 * SY * W + mi], m8 = cbuf[8 * SY * W + mi],
                        m9 = cbuf[9 * SY * W + mi];
            sg1[r * SX + c] = m6 * d0 + m7 * d1;
            sg1[TTY * SX + r * SX + c] = m8 * d0 + m9 * d1;
        };
        auto ex_at = [&](int r, int ii) {          // ii = i + Q
            const int col = ii - Q + TXOFF;
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                const float* bl = cbuf + f * SY * W + (r + Q) * W + col;
                auto Bf = [&](int k) { return bl[k]; };
#pragma unroll
                for (int m = 1; m <= Q; ++m)
                    sex[((f * Q + (m - 1)) * TTY + r) * EX + ii] =
                        (ii + edge_lo<O>(m) >= 0) ? Edge<O>::template e<float>(m, Bf) : 0.f;
            }
        };
        for (int task = ty; task < T_END; task += 8) {
            if (task < T_G1H) {
                g1_at(task - T_G1, tx + Q);
            } else if (task < T_G2) {
                const int lane = (task - T_G1H) * 32 + tx;
                if (lane < TTY * 2 * Q) {
                    const int r = lane / (2 * Q), h = lane - r * (2 * Q);
                    g1_at(r, h < Q ? h : TTX + h);
                }
            } else if (task < T_EX) {
                const int r = task - T_G2;
                const int col = tx + TXOFF;
                const float* p0 = su + r * W + col;
                const float* p1 = p0 + SY * W;
                float d0 = 0.f, d1 = 0.f;
#pragma unroll
                for (int k = 1; k <= Q; ++k) {
                    d0 += ak[k - 1] * (p0[k] - p0[-k]);
                    d1 += ak[k - 1] * (p1[k] - p1[-k]);
                }
                d0 *= ih1;
                d1 *= ih1;
                const int mi = r * W + col;
                const float m6 = cbuf[6 * SY * W + mi], m7 = cbuf[7 * SY * W + mi], m8 = cbuf[8 * SY * W + mi],
                            m9 = cbuf[9 * SY * W + mi];
                sg2[r * TTX + tx] = m6 * d0 + m8 * d1;
                sg2[SY * TTX + r * TTX + tx] = m7 * d0 + m9 * d1;
            } else if (task < T_EXH) {
                ex_at(task - T_EX, tx + Q);
            } else if (task < T_EY) {
                const int lane = (task - T_EXH) * 32 + tx;
                if (lane < TTY * Q) {
                    const int r = lane / Q, ii = lane - r * Q;
                    ex_at(r, ii);
                }
            } else {
                const int jj = task - T_EY;        // j = jj - Q
                const int col = tx + TXOFF;
#pragma unroll
                for (int f = 0; f < 3; ++f) {
                    const float* bl = cbuf + (3 + f) * SY * W + jj * W + col;
                    auto Bf = [&](int k) { return bl[k * W]; };
#pragma unroll
                    for (int m = 1; m <= Q; ++m)
                        sey[((f * Q + (m - 1)) * EY + jj) * TTX + tx] =
                            (jj + edge_lo<O>(m) >= 0) ? Edge<O>::template e<float>(m, Bf) : 0.f;
                }
            }
        }
        __syncthreads();
        // the coefficient tile is consumed: prefetch the next tile (coefficients and the other
        // displacement stage) while this tile's outputs are formed
        const int next = tile + gridDim.x;
        if (threadIdx.x == 0 && next < ntiles) {
            fence_proxy_async();
            issue(next, s ^ 1, true);
        }
        // ---- phase 3: outputs at rows pr0 and pr0 + 1 of column tx
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int r = pr0 + k;
            if (!act[k]) continue;
            const int gy = y0 + r;
            const float* u0 = su + (r + Q) * W + tx + TXOFF;
            const float* u1 = u0 + SY * W;
            const float uc0 = u0[0], uc1 = u1[0];
            float rx0 = 0.f, rx1 = 0.f, ry0 = 0.f, ry1 = 0.f;
#pragma unroll
            for (int m = 1; m <= Q; ++m) {
                const float* ex0 = sex + ((0 * Q + (m - 1)) * TTY + r) * EX + (tx + Q);
                const float* ex1 = ex0 + Q * TTY * EX;
                const float* ex2 = ex1 + Q * TTY * EX;
                const float dp0 = u0[m] - uc0, dp1 = u1[m] - uc1, dm0 = u0[-m] - uc0, dm1 = u1[-m] - uc1;
                rx0 += ex0[0] * dp0 + ex1[0] * dp1 + ex0[-m] * dm0 + ex1[-m] * dm1;
                rx1 += ex1[0] * dp0 + ex2[0] * dp1 + ex1[-m] * dm0 + ex2[-m] * dm1;
                const float* ey0 = sey + ((0 * Q + (m - 1)) * EY + (r + Q)) * TTX + tx;
                const float* ey1 = ey0 + Q * EY * TTX;
                const float* ey2 = ey1 + Q * EY * TTX;
                const float qp0 = u0[m * W] - uc0, qp1 = u1[m * W] - uc1, qm0 = u0[-m * W] - uc0,
                            qm1 = u1[-m * W] - uc1;
                ry0 += ey0[0] * qp0 + ey1[0] * qp1 + ey0[-m * TTX] * qm0 + ey1[-m * TTX] * qm1;
                ry1 += ey1[0] * qp0 + ey2[0] * qp1 + ey1[-m * TTX] * qm0 + ey2[-m * TTX] * qm1;
            }
            float r0 = rx0 * ih11 + ry0 * ih22;
            float r1 = rx1 * ih11 + ry1 * ih22;
            const float* g10 = sg1 + r * SX + (tx + Q);
            const float* g11 = g10 + TTY * SX;
            const float* g20 = sg2 + (r + Q) * TTX + tx;
            const float* g21 = g20 + SY * TTX;
            float m10 = 0.f, m11 = 0.f, m20 = 0.f, m21 = 0.f;
#pragma unroll
            for (int kk = 1; kk <= Q; ++kk) {
                m10 += ak[kk - 1] * (g10[kk] - g10[-kk]);
                m11 += ak[kk - 1] * (g11[kk] - g11[-kk]);
                m20 += ak[kk - 1] * (g20[kk * TTX] - g20[-kk * TTX]);
                m21 += ak[kk - 1] * (g21[kk * TTX] - g21[-kk * TTX]);
            }
            r0 += m10 * ih1 + m20 * ih2;
            r1 += m11 * ih1 + m21 * ih2;
            const size_t gi = (size_t)gy * P + gx;
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
                Un[gi] = 2.f * uc0 - up0[k] + dt2 * wv[k] * r0;
                Un[gi + plane] = 2.f * uc1 - up1[k] + dt2 * wv[k] * r1;
            } else {
                float* __restrict__ R = reinterpret_cast<float*>(B.r);
                R[gi] = r0;
                R[gi + plane] = r1;
            }
        }
        __syncthreads();   // phase-2 buffers and this displacement stage are reused next round
    }
}

}  // namespace sbp
