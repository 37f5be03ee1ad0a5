// libsbp 3-D operator kernels: one curvilinear block of n1 x n2 x n3 nodes (the d = 3 form of
// Sec. 3.3, 4.3-4.7 and 5).  A leapfrog step is three kernel families:
//   k3_flux  -- the mixed fluxes q_ij = sum_{k != i} c_ijkl D_k u_l (9 fields) from u^n;
//   k3_div   -- r_j = sum_i D_i q_ij + sum_i D_ii^FC(c_ijil) u_l, then the leapfrog store;
//   k3_face  -- the traction / displacement SATs of the two faces x_m = 0, 1 (one launch per m),
//               added to the stored step (they are linear in r, so they can follow k3_div).
// Layout: every scalar field is [n3][n2][pitch] in the arithmetic type T, pitch = n1 rounded up
// to 128 bytes; field f of a group starts at f * fs (fs = n3 * n2 * pitch).
//   cm: 27 fields, M^{ik}_{jl} = c_ijkl for the pairs (i, k) = (1,2), (1,3), (2,3), field 9p + 3j + l
//       (the other ordering is its transpose: c_kjil = c_ilkj by major symmetry);
//   cd: 18 fields, c_ijil of direction i as a symmetric 3 x 3 (jl = 11 12 13 22 23 33), field 6i + s;
//   w : 1 / (rho J).
#pragma once
#include "sbp_device.cuh"

namespace sbp3 {
using namespace sbp;

constexpr int BC_DISPLACEMENT = 0, BC_TRACTION = 1;

struct Grid3 {
    int n[3];               // nodes along x1, x2, x3
    long long s[3];         // element strides along x1, x2, x3 (1, pitch, n2 * pitch)
    long long fs;           // field stride (elements)
    double ih[3];           // 1 / h_i
};

__device__ __forceinline__ int sym3(int j, int l) {
    // index of (j, l) in 11 12 13 22 23 33
    const int a = j < l ? j : l, b = j < l ? l : j;
    return a == 0 ? b : (a == 1 ? 2 + b : 5);
}
// pair index of (i, k), i < k: (0,1) -> 0, (0,2) -> 1, (1,2) -> 2
__host__ __device__ __forceinline__ constexpr int pair3(int i, int k) { return i + k - 1; }

template <typename T> __device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

// c_ijkl at element offset o from the stored 45 fields
template <typename T>
__device__ __forceinline__ T cfull(const T* __restrict__ cm, const T* __restrict__ cd, long long fs, int i, int j,
                                   int k, int l, long long o) {
    if (i == k) return ldg(cd + (long long)(6 * i + sym3(j, l)) * fs + o);
    if (i < k) return ldg(cm + (long long)(9 * pair3(i, k) + 3 * j + l) * fs + o);
    return ldg(cm + (long long)(9 * pair3(k, i) + 3 * l + j) * fs + o);
}

// ------------------------------------------------------------------ narrow D_xx^FC for 3 components
// r_j += h^2 sum_l D_xx^FC(b_jl) u_l along one grid line; u(l, t) and b(s, t) read index t of
// the line, b symmetric with s = sym3(j, l).  Closure rows from the coefficient table, interior
// rows through the edge weights E_m (the same splitting as the 2-component rows).
template <int O, typename T, class FU, class FB>
__device__ __forceinline__ void dxx3(int N, int i, FU u, FB b, T r[3]) {
    using P = Ord<O>;
    if (i < P::NCLOS || i >= N - P::NCLOS) {
        const bool right = i >= N - P::NCLOS;
        const int row = right ? N - 1 - i : i;
        for (int t = P::cstart(row); t < P::cstart(row + 1); ++t) {
            int j = P::cj(t), k = P::ck(t);
            if (right) { j = N - 1 - j; k = N - 1 - k; }
            const T c = P::template ccT<T>(t);
            const T b00 = b(0, k), b01 = b(1, k), b02 = b(2, k), b11 = b(3, k), b12 = b(4, k), b22 = b(5, k);
            const T u0 = u(0, j), u1 = u(1, j), u2 = u(2, j);
            r[0] += c * (b00 * u0 + b01 * u1 + b02 * u2);
            r[1] += c * (b01 * u0 + b11 * u1 + b12 * u2);
            r[2] += c * (b02 * u0 + b12 * u1 + b22 * u2);
        }
    } else {
        const T uc0 = u(0, i), uc1 = u(1, i), uc2 = u(2, i);
#pragma unroll
        for (int m = 1; m <= P::Q; ++m) {
            T ep[6], em[6];
#pragma unroll
            for (int s = 0; s < 6; ++s) {
                ep[s] = Edge<O>::template e<T>(m, [&](int k) { return b(s, i + k); });
                em[s] = Edge<O>::template e<T>(m, [&](int k) { return b(s, i - m + k); });
            }
            const T p0 = u(0, i + m) - uc0, p1 = u(1, i + m) - uc1, p2 = u(2, i + m) - uc2;
            const T m0 = u(0, i - m) - uc0, m1 = u(1, i - m) - uc1, m2 = u(2, i - m) - uc2;
            r[0] += ep[0] * p0 + ep[1] * p1 + ep[2] * p2 + em[0] * m0 + em[1] * m1 + em[2] * m2;
            r[1] += ep[1] * p0 + ep[3] * p1 + ep[4] * p2 + em[1] * m0 + em[3] * m1 + em[4] * m2;
            r[2] += ep[2] * p0 + ep[4] * p1 + ep[5] * p2 + em[2] * m0 + em[4] * m1 + em[5] * m2;
        }
    }
}

constexpr int BX = 32, BY = 8;

// ------------------------------------------------------------------ mixed fluxes
template <typename T, int O>
__global__ void __launch_bounds__(BX * BY) k3_flux(Grid3 g, const T* __restrict__ u, const T* __restrict__ cm,
                                                   T* __restrict__ q) {
    const int i1 = blockIdx.x * BX + threadIdx.x, i2 = blockIdx.y * BY + threadIdx.y, i3 = blockIdx.z;
    if (i1 >= g.n[0] || i2 >= g.n[1]) return;
    const int idx[3] = {i1, i2, i3};
    const long long o = i1 + i2 * g.s[1] + i3 * g.s[2];
    T gr[3][3];                                   // gr[k][l] = D_k u_l
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const T ihk = T(g.ih[k]);
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            const T* line = u + l * g.fs + o - idx[k] * g.s[k];
            const long long sk = g.s[k];
            gr[k][l] = ihk * dsum<O, T>(g.n[k], idx[k], [&](int t) { return ldg(line + t * sk); });
        }
    }
    T qq[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) qq[i][j] = T(0);
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const int i = p == 2 ? 1 : 0, k = p == 0 ? 1 : 2;
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                const T M = ldg(cm + (long long)(9 * p + 3 * j + l) * g.fs + o);
                qq[i][j] += M * gr[k][l];             // c_ijkl D_k u_l
                qq[k][l] += M * gr[i][j];             // c_klij D_i u_j (= c_kl ij, major symmetry)
            }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) q[(long long)(3 * i + j) * g.fs + o] = qq[i][j];
}

// ------------------------------------------------------------------ divergence and leapfrog store
// MODE 0: leapfrog in increment form, d = du + dt^2 w r, un = u + d (du updated in place);
// MODE 1: apply, out = w r.
template <typename T, int O, int MODE>
__global__ void __launch_bounds__(BX * BY) k3_div(Grid3 g, const T* __restrict__ u, const T* __restrict__ q,
                                                  const T* __restrict__ cd, const T* __restrict__ w,
                                                  T* __restrict__ du, T* __restrict__ un, T dt2) {
    const int i1 = blockIdx.x * BX + threadIdx.x, i2 = blockIdx.y * BY + threadIdx.y, i3 = blockIdx.z;
    if (i1 >= g.n[0] || i2 >= g.n[1]) return;
    const int idx[3] = {i1, i2, i3};
    const long long o = i1 + i2 * g.s[1] + i3 * g.s[2];
    T r[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const T ihi = T(g.ih[i]);
        const long long si = g.s[i];
        const long long base = o - idx[i] * si;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const T* line = q + (long long)(3 * i + j) * g.fs + base;
            r[j] += ihi * dsum<O, T>(g.n[i], idx[i], [&](int t) { return ldg(line + t * si); });
        }
        T rr[3] = {T(0), T(0), T(0)};
        const T* cdi = cd + (long long)(6 * i) * g.fs + base;
        const T* ul = u + base;
        const long long fs = g.fs;
        dxx3<O, T>(g.n[i], idx[i], [&](int l, int t) { return ldg(ul + l * fs + t * si); },
                   [&](int s, int t) { return ldg(cdi + s * fs + t * si); }, rr);
        const T ih2 = ihi * ihi;
#pragma unroll
        for (int j = 0; j < 3; ++j) r[j] += ih2 * rr[j];
    }
    const T wv = ldg(w + o);
    if constexpr (MODE == 0) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const long long oj = j * g.fs + o;
            const T d = du[oj] + dt2 * wv * r[j];
            du[oj] = d;
            un[oj] = ldg(u + oj) + d;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 3; ++j) un[j * g.fs + o] = wv * r[j];
    }
}

// ------------------------------------------------------------------ boundary SATs of the faces x_m = 0, 1
// One thread per face node (a, b) along the two tangential directions (p < t), blockIdx.z = side.
//   traction:     J SAT_J = -H^-1 P_f nu c_mJkL D_k u_L              (face node only)
//   displacement: J SAT_J = H^-1 [ sum_k D_k^T (nu c_mLkJ P_f u_L) - P_f (beta d / h1) c_mJmL u_L ]
// H^-1 P_f is 1 / (h_m hw_0) at a face node; D_m^T spreads the normal term over the first NCOL
// nodes of the normal line (H^-1 D_m^T at depth t: D_m[face][t] / (h_m hw_t)); the tangential
// D_k^T stays on the face, weighted by hw_k(a') / hw_k(a).  MODE 0 adds dt^2 w SAT to du and un,
// MODE 1 adds w SAT to the applied field.
template <typename T, int O, int MODE>
__global__ void __launch_bounds__(128) k3_face(Grid3 g, int m, int kind0, int kind1, double beta,
                                               const T* __restrict__ u, const T* __restrict__ cm,
                                               const T* __restrict__ cd, const T* __restrict__ w,
                                               T* __restrict__ du, T* __restrict__ un, T dt2) {
    using P = Ord<O>;
    const int pd = m == 0 ? 1 : 0, td = m == 2 ? 1 : 2;
    const int a = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y * blockDim.y + threadIdx.y;
    const int side = blockIdx.z;
    if (a >= g.n[pd] || b >= g.n[td]) return;
    const int kind = side ? kind1 : kind0;
    const int Nm = g.n[m];
    const int im = side ? Nm - 1 : 0;
    const T nu = side ? T(1) : T(-1);
    int idx[3];
    idx[m] = im;
    idx[pd] = a;
    idx[td] = b;
    const long long o = idx[0] + idx[1] * g.s[1] + idx[2] * g.s[2];
    const long long fs = g.fs;
    const T ihb = T(g.ih[m] / hweight<O>(Nm, im));        // H^-1 P_f at the face node
    T rs[3] = {T(0), T(0), T(0)};
    if (kind == BC_TRACTION) {
        T gr[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const T ihk = T(g.ih[k]);
            const long long sk = g.s[k];
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                const T* line = u + l * fs + o - idx[k] * sk;
                gr[k][l] = ihk * dsum<O, T>(g.n[k], idx[k], [&](int t) { return ldg(line + t * sk); });
            }
        }
#pragma unroll
        for (int J = 0; J < 3; ++J) {
            T s = T(0);
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int L = 0; L < 3; ++L) s += cfull(cm, cd, fs, m, J, k, L, o) * gr[k][L];
            rs[J] = -ihb * nu * s;
        }
    } else {
        T uf[3];
#pragma unroll
        for (int L = 0; L < 3; ++L) uf[L] = ldg(u + L * fs + o);
        // penalty -H^-1 P_f (beta d / h1) c_mJmL u_L, h1 = h_m hw_0
        const T pen = T(beta * 3.0) * ihb * ihb;
#pragma unroll
        for (int J = 0; J < 3; ++J) {
            T s = T(0);
#pragma unroll
            for (int L = 0; L < 3; ++L) s += cfull(cm, cd, fs, m, J, m, L, o) * uf[L];
            rs[J] = -pen * s;
        }
        // tangential transposes
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            const int k = kk ? td : pd;
            const int Nk = g.n[k], ak = idx[k];
            const long long sk = g.s[k];
            const int W = P::NCOL - 1 > P::Q ? P::NCOL - 1 : P::Q;
            const int lo = ak - W < 0 ? 0 : ak - W, hi = ak + W > Nk - 1 ? Nk - 1 : ak + W;
            const T iwa = T(1.0 / hweight<O>(Nk, ak));
            for (int a2 = lo; a2 <= hi; ++a2) {
                const T dc = dcoefT<O, T>(Nk, a2, ak);
                if (dc == T(0)) continue;
                const T coef = ihb * T(g.ih[k]) * dc * hweightT<O, T>(Nk, a2) * iwa * nu;
                const long long o2 = o + (long long)(a2 - ak) * sk;
                T v[3];
#pragma unroll
                for (int L = 0; L < 3; ++L) v[L] = ldg(u + L * fs + o2);
#pragma unroll
                for (int J = 0; J < 3; ++J) {
                    T s = T(0);
#pragma unroll
                    for (int L = 0; L < 3; ++L) s += cfull(cm, cd, fs, m, L, k, J, o2) * v[L];
                    rs[J] += coef * s;
                }
            }
        }
        // normal transpose: depth t = 0 .. NCOL-1 along the normal line
        T vn[3];
#pragma unroll
        for (int J = 0; J < 3; ++J) {
            T s = T(0);
#pragma unroll
            for (int L = 0; L < 3; ++L) s += cfull(cm, cd, fs, m, L, m, J, o) * uf[L];
            vn[J] = nu * s;
        }
        const T ihm = T(g.ih[m]);
        for (int t = 0; t < P::NCOL; ++t) {
            const int col = side ? Nm - 1 - t : t;
            const T dc = dcoefT<O, T>(Nm, im, col);
            if (dc == T(0)) continue;
            const T coef = ihm * ihm * dc / hweightT<O, T>(Nm, col);
            const long long on = o + (long long)(col - im) * g.s[m];
            const T wv = ldg(w + on);
            if (t == 0) {
#pragma unroll
                for (int J = 0; J < 3; ++J) rs[J] += coef * vn[J];
                continue;
            }
#pragma unroll
            for (int J = 0; J < 3; ++J) {
                const long long oj = J * fs + on;
                if constexpr (MODE == 0) {
                    const T dlt = dt2 * wv * coef * vn[J];
                    du[oj] += dlt;
                    un[oj] += dlt;
                } else {
                    un[oj] += wv * coef * vn[J];
                }
            }
        }
    }
    const T wv = ldg(w + o);
#pragma unroll
    for (int J = 0; J < 3; ++J) {
        const long long oj = J * fs + o;
        if constexpr (MODE == 0) {
            const T dlt = dt2 * wv * rs[J];
            du[oj] += dlt;
            un[oj] += dlt;
        } else {
            un[oj] += wv * rs[J];
        }
    }
}

// ------------------------------------------------------------------ setup: metric and material
// For the x3-planes k0 <= i3 < k0 + nk: G_iI = D_i X_I (FP64), J = det G, F = G^-1,
// c_ijkl = J F_Ii C_IjKl F_Kk for the 45 stored entries, w = 1 / (rho J).  rho and C45 are the
// compact host layout of those planes (C45 entry t = 9p - p(p-1)/2 + (q - p), p = 3I+J <= q = 3K+L).
__host__ __device__ __forceinline__ constexpr int tri45(int p, int q) {
    return p <= q ? 9 * p - p * (p - 1) / 2 + (q - p) : 9 * q - q * (q - 1) / 2 + (p - q);
}

template <typename T, int O>
__global__ void __launch_bounds__(128) k3_material(Grid3 g, const double* __restrict__ X, int k0, int nk,
                                                   const double* __restrict__ rho, const double* __restrict__ C45,
                                                   T* __restrict__ cm, T* __restrict__ cd, T* __restrict__ w,
                                                   int* __restrict__ err) {
    const int i1 = blockIdx.x * blockDim.x + threadIdx.x, i2 = blockIdx.y, kk = blockIdx.z;
    if (i1 >= g.n[0] || i2 >= g.n[1] || kk >= nk) return;
    const int i3 = k0 + kk;
    const int idx[3] = {i1, i2, i3};
    const long long o = i1 + i2 * g.s[1] + i3 * g.s[2];
    double G[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const long long si = g.s[i];
#pragma unroll
        for (int I = 0; I < 3; ++I) {
            const double* line = X + I * g.fs + o - idx[i] * si;
            G[i][I] = g.ih[i] * dsum<O, double>(g.n[i], idx[i], [&](int t) { return line[t * si]; });
        }
    }
    const double J = G[0][0] * (G[1][1] * G[2][2] - G[1][2] * G[2][1]) -
                     G[0][1] * (G[1][0] * G[2][2] - G[1][2] * G[2][0]) +
                     G[0][2] * (G[1][0] * G[2][1] - G[1][1] * G[2][0]);
    if (!(J > 0.0)) {
        atomicExch(err, 1);
        return;
    }
    // F_Ii = (G^-1)_Ii = cof(G)_iI / J
    double F[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int I = 0; I < 3; ++I) {
            const int i1c = (i + 1) % 3, i2c = (i + 2) % 3, I1 = (I + 1) % 3, I2 = (I + 2) % 3;
            F[I][i] = (G[i1c][I1] * G[i2c][I2] - G[i1c][I2] * G[i2c][I1]) / J;
        }
    const long long np = (long long)g.n[0] * g.n[1];
    const long long hc = (long long)kk * np + (long long)i2 * g.n[0] + i1;     // compact index
    const long long cstr = (long long)nk * np;
    double Cn[45];
#pragma unroll
    for (int t = 0; t < 45; ++t) Cn[t] = C45[t * cstr + hc];
    auto cval = [&](int i, int j, int k, int l) {
        double s = 0.0;
#pragma unroll
        for (int I = 0; I < 3; ++I) {
            double sI = 0.0;
#pragma unroll
            for (int K = 0; K < 3; ++K) sI += Cn[tri45(3 * I + j, 3 * K + l)] * F[K][k];
            s += F[I][i] * sI;
        }
        return J * s;
    };
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int l = j; l < 3; ++l) cd[(long long)(6 * i + sym3(j, l)) * g.fs + o] = T(cval(i, j, i, l));
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const int i = p == 2 ? 1 : 0, k = p == 0 ? 1 : 2;
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int l = 0; l < 3; ++l) cm[(long long)(9 * p + 3 * j + l) * g.fs + o] = T(cval(i, j, k, l));
    }
    w[o] = T(1.0 / (rho[hc] * J));
}

// ------------------------------------------------------------------ state conversion
// compact FP64 (3 components) <-> pitched T.  Load: u_cur, u_prev and the increment
// u_cur - u_prev formed in FP64.  Store: the two levels back to FP64.
template <typename T>
__global__ void k3_load_state(Grid3 g, const double* __restrict__ prev, const double* __restrict__ cur,
                              T* __restrict__ up, T* __restrict__ uc, T* __restrict__ du) {
    const int i1 = blockIdx.x * blockDim.x + threadIdx.x, i2 = blockIdx.y, i3 = blockIdx.z;
    if (i1 >= g.n[0]) return;
    const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
    const long long hc = ((long long)i3 * g.n[1] + i2) * g.n[0] + i1;
    const long long o = i1 + i2 * g.s[1] + i3 * g.s[2];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double a = prev[c * N + hc], b = cur[c * N + hc];
        up[c * g.fs + o] = T(a);
        uc[c * g.fs + o] = T(b);
        du[c * g.fs + o] = T(b - a);
    }
}

template <typename T>
__global__ void k3_store_field(Grid3 g, const T* __restrict__ f, double* __restrict__ out) {
    const int i1 = blockIdx.x * blockDim.x + threadIdx.x, i2 = blockIdx.y, i3 = blockIdx.z;
    if (i1 >= g.n[0]) return;
    const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
    const long long hc = ((long long)i3 * g.n[1] + i2) * g.n[0] + i1;
    const long long o = i1 + i2 * g.s[1] + i3 * g.s[2];
#pragma unroll
    for (int c = 0; c < 3; ++c) out[c * N + hc] = double(f[c * g.fs + o]);
}

template <typename T>
__global__ void k3_load_field(Grid3 g, const double* __restrict__ in, T* __restrict__ f) {
    const int i1 = blockIdx.x * blockDim.x + threadIdx.x, i2 = blockIdx.y, i3 = blockIdx.z;
    if (i1 >= g.n[0]) return;
    const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
    const long long hc = ((long long)i3 * g.n[1] + i2) * g.n[0] + i1;
    const long long o = i1 + i2 * g.s[1] + i3 * g.s[2];
#pragma unroll
    for (int c = 0; c < 3; ++c) f[c * g.fs + o] = T(in[c * N + hc]);
}

}  // namespace sbp3
