// Wide-stencil variant of the spatial operator (the comparison of Sec. 7.1): every term of
//   r_j = sum_{i,k} D_i (c_ijkl D_k u_l)
// is a first-derivative SBP operator applied twice, the narrow D_xx^FC(b) of the main scheme
// replaced by D b D -- the same SBP form H D b D = -D^T H b D + B b D without the remainder R(b),
// so the operator is fully compatible as well -- and the SATs are exactly those of the narrow
// scheme.  Two passes over each block:
//   k_wide_flux: the fluxes G_ij = sum_{k,l} c_ijkl D_k u_l at every node (boundary rows of D at the
//                faces), 4 planes G_10, G_11, G_20, G_21;
//   k_wide_div:  r_j = D_1 G_1j + D_2 G_2j + the SAT terms of k_face_sat + J f, and the step epilogue
//                (leapfrog update, operator output or RK4 stage).
#pragma once
#include "sbp_kernels.cuh"

namespace sbp {

template <typename T, int O>
__global__ void k_wide_flux(BlockDev B, StepArgs a, T* __restrict__ G) {
    const long long n = (long long)B.n1 * B.n2;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int i2 = (int)(t / B.n1), i1 = (int)(t - (long long)i2 * B.n1);
    const int P = B.pitch;
    const size_t plane = (size_t)B.n2 * P, gi = (size_t)i2 * P + i1;
    const T* __restrict__ U0 = reinterpret_cast<const T*>(B.u[a.cur]);
    const T* __restrict__ U1 = U0 + plane;
    const T* __restrict__ C = reinterpret_cast<const T*>(B.c);
    const T ih1 = ih1T<T>(B), ih2 = ih2T<T>(B);
    const T d10 = dsum<O, T>(B.n1, i1, [&](int aa) { return U0[(size_t)i2 * P + aa]; }) * ih1;
    const T d11 = dsum<O, T>(B.n1, i1, [&](int aa) { return U1[(size_t)i2 * P + aa]; }) * ih1;
    const T d20 = dsum<O, T>(B.n2, i2, [&](int bb) { return U0[(size_t)bb * P + i1]; }) * ih2;
    const T d21 = dsum<O, T>(B.n2, i2, [&](int bb) { return U1[(size_t)bb * P + i1]; }) * ih2;
    T c[10];
#pragma unroll
    for (int p = 0; p < 10; ++p) c[p] = C[p * plane + gi];
    // planes: 0 c0000 1 c0001 2 c0101 | 3 c1010 4 c1011 5 c1111 | 6 c0010 7 c0011 8 c0110 9 c0111,
    // with c_ijkl = c_klij for the entries not stored
    G[gi] = c[0] * d10 + c[1] * d11 + c[6] * d20 + c[7] * d21;                  // G_10
    G[plane + gi] = c[1] * d10 + c[2] * d11 + c[8] * d20 + c[9] * d21;          // G_11
    G[2 * plane + gi] = c[6] * d10 + c[8] * d11 + c[3] * d20 + c[4] * d21;      // G_20
    G[3 * plane + gi] = c[7] * d10 + c[9] * d11 + c[4] * d20 + c[5] * d21;      // G_21
}

template <typename T, int O, int MODE>
__global__ void k_wide_div(BlockDev B, StepArgs a, const T* __restrict__ G) {
    const long long n = (long long)B.n1 * B.n2;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int n1 = B.n1, n2 = B.n2;
    const int i2 = (int)(t / n1), i1 = (int)(t - (long long)i2 * n1);
    const int P = B.pitch;
    const size_t plane = (size_t)n2 * P, gi = (size_t)i2 * P + i1;
    const T ih1 = ih1T<T>(B), ih2 = ih2T<T>(B);
    T r0 = dsum<O, T>(n1, i1, [&](int aa) { return G[(size_t)i2 * P + aa]; }) * ih1 +
           dsum<O, T>(n2, i2, [&](int bb) { return G[2 * plane + (size_t)bb * P + i1]; }) * ih2;
    T r1 = dsum<O, T>(n1, i1, [&](int aa) { return G[plane + (size_t)i2 * P + aa]; }) * ih1 +
           dsum<O, T>(n2, i2, [&](int bb) { return G[3 * plane + (size_t)bb * P + i1]; }) * ih2;
    // SAT terms (k_face_sat): the face term at the face node, the D_m^T spread into the first
    // NCOL nodes along the normal
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const FaceDev& F = B.f[f];
        const int m = F.m;
        const int im = m == 0 ? i1 : i2, Nm = m == 0 ? n1 : n2;
        const int d = F.side ? Nm - 1 - im : im;
        if (d >= Ord<O>::NCOL) continue;
        const int s = m == 0 ? i2 : i1;
        const T* __restrict__ sat = reinterpret_cast<const T*>(F.sat);
        const int nf = F.nf;
        const T fac = facT<T>(F, d);
        r0 += fac * sat[2 * nf + s];
        r1 += fac * sat[3 * nf + s];
        if (d == 0) {
            r0 += sat[s];
            r1 += sat[nf + s];
        }
    }
    if (a.with_data && B.jf) {
        const T* __restrict__ JF = reinterpret_cast<const T*>(B.jf);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (k >= a.K) break;
            r0 += T(a.Tk[k]) * JF[(size_t)k * plane + gi];
            r1 += T(a.Tk[k]) * JF[(size_t)(a.K + k) * plane + gi];
        }
    }
    T dd00, dd01, dd11;
    const bool damped = MODE != 1 && robin_damping_at<T>(B, i1, i2, dd00, dd01, dd11);
    if (MODE == 0) {
        const T* __restrict__ U = reinterpret_cast<const T*>(B.u[a.cur]);
        leapfrog_store<T>(B, a, gi, plane, U[gi], U[gi + plane], reinterpret_cast<const T*>(B.w)[gi], r0, r1, damped,
                          dd00, dd01, dd11);
    } else if (MODE == 2) {
        if (damped) {
            T v0, v1;
            rk4_stage_velocity<T>(B, a, gi, plane, v0, v1);
            r0 -= dd00 * v0 + dd01 * v1;
            r1 -= dd01 * v0 + dd11 * v1;
        }
        rk4_store<T>(B, a, gi, plane, reinterpret_cast<const T*>(B.w)[gi], r0, r1);
    } else {
        T* __restrict__ R = reinterpret_cast<T*>(B.r);
        R[gi] = r0;
        R[gi + plane] = r1;
    }
}

}  // namespace sbp
