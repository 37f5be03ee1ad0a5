// libsbp 3-D operator kernels: one curvilinear block of n1 x n2 x n3 nodes (the d = 3 form of
// Sec. 3.3, 4.3-4.7 and 5).  A leapfrog step is three kernel families:
//   k3_flux  -- the mixed fluxes q_ij = sum_{k != i} c_ijkl D_k u_l (9 fields) from u^n;
//   k3_div_int / k3_div_shell -- r_j = sum_i D_i q_ij + sum_i D_ii^FC(c_ijil) u_l, then the leapfrog
//               store (MODE 0: increment form, d = du + dt^2 w r, un = u + d; MODE 1: out = w r),
//               on the x1-interior columns at every i2, i3 (with the x2 / x3 face SATs) and on the
//               x1 slabs near the x1 faces (with every face SAT that reaches the node).
// Layout: every scalar field is [n3][n2][pitch] in the arithmetic type T, pitch = n1 rounded up
// to 128 bytes; field f of a group starts at f * fs (fs = n3 * n2 * pitch).
//   cm: 27 fields, M^{ik}_{jl} = c_ijkl for the pairs (i, k) = (1,2), (1,3), (2,3), field 9p + 3j + l
//       (the other ordering is its transpose: c_kjil = c_ilkj by major symmetry);
//   cd: 18 fields, c_ijil of direction i as a symmetric 3 x 3 (jl = 11 12 13 22 23 33), field 6i + s;
//   w : 1 / (rho J).
#pragma once
#include <utility>

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
// the line, b symmetric with s = sym3(j, l).  Closure rows come from the coefficient table.  An
// interior row is sum_m E_m(i) (u_{i+m} - u_i) + E_m(i-m) (u_{i-m} - u_i) with the edge weights
// E_m(i) = sum_t e_{m,t} b_{i+t}; collecting the terms of each b_{i+k} (k = -Q..Q) gives
//   h^2 D_xx(b) u |_i = sum_k b_{i+k} L_k(u),  L_k(u) = sum_m e_{m,k} (u_{i+m} - u_i) + e_{m,k+m} (u_{i-m} - u_i),
// so every b value of the window is read once and the e's fold into compile-time constants.
template <int O, typename T> __device__ __forceinline__ T edge_wT(int m, int kk) {
    return Edge<O>::template e<T>(m, [&](int q) { return q == kk ? T(1) : T(0); });
}

// Closure rows of D_xx^FC, unrolled at compile time.  Row ROW of the table is a list of terms
// c_t b(k_t) u(j_t); grouping them by k gives r_j += sum_k sum_l b_jl(k) V_k(u_l) with
// V_k(u) = sum_{t: k_t = k} c_t u(j_t), so the u window (NCLOSJ columns) and each b column are
// read once and every c_t, j_t, k_t is a constant.
namespace tab {
#define SBP_TABLE static constexpr
#include "sbp_tables.inc"
#undef SBP_TABLE
}  // namespace tab

template <int O> struct CTab;
#define SBP3_CTAB(O)                                                                                   \
    template <> struct CTab<O> {                                                                       \
        static constexpr int NCLOS = SBP##O##_NCLOS, NJ = SBP##O##_NCLOSJ;                             \
        static constexpr const int* start = tab::sbp##O##_CLOS_START;                                  \
        static constexpr const int* cj = tab::sbp##O##_CLOS_J;                                         \
        static constexpr const int* ck = tab::sbp##O##_CLOS_K;                                         \
        static constexpr const double* cc = tab::sbp##O##_CLOS_C;                                      \
    };
SBP3_CTAB(2)
SBP3_CTAB(4)
SBP3_CTAB(6)
#undef SBP3_CTAB

template <int O> constexpr bool clos_has_k(int row, int k) {
    for (int t = CTab<O>::start[row]; t < CTab<O>::start[row + 1]; ++t)
        if (CTab<O>::ck[t] == k) return true;
    return false;
}

template <int O, int ROW, int K, typename T, int... I>
__device__ __forceinline__ void clos_vk(const T (&uw)[3][CTab<O>::NJ], T V[3], std::integer_sequence<int, I...>) {
    constexpr int T0 = CTab<O>::start[ROW];
    (
        [&] {
            if constexpr (CTab<O>::ck[T0 + I] == K) {
                constexpr int j = CTab<O>::cj[T0 + I];
                const T c = T(CTab<O>::cc[T0 + I]);
                V[0] += c * uw[0][j];
                V[1] += c * uw[1][j];
                V[2] += c * uw[2][j];
            }
        }(),
        ...);
}

template <int O, int ROW, typename T, class FB, int... K>
__device__ __forceinline__ void clos_row_k(const T (&uw)[3][CTab<O>::NJ], FB b, T r[3],
                                           std::integer_sequence<int, K...>) {
    constexpr int NT = CTab<O>::start[ROW + 1] - CTab<O>::start[ROW];
    (
        [&] {
            if constexpr (clos_has_k<O>(ROW, K)) {
                T V[3] = {T(0), T(0), T(0)};
                clos_vk<O, ROW, K>(uw, V, std::make_integer_sequence<int, NT>());
                const T b00 = b(0, K), b01 = b(1, K), b02 = b(2, K), b11 = b(3, K), b12 = b(4, K), b22 = b(5, K);
                r[0] += b00 * V[0] + b01 * V[1] + b02 * V[2];
                r[1] += b01 * V[0] + b11 * V[1] + b12 * V[2];
                r[2] += b02 * V[0] + b12 * V[1] + b22 * V[2];
            }
        }(),
        ...);
}

// one closure row, shared by the three directions and both ends: the node's pointers up (u) and
// cp (the 6 narrow coefficients of the direction), column c of the line (counted from the nearer
// end) at offset (c - ROW) * Ss from the node, Ss = +stride at the left end and -stride at the right
template <int O, int ROW, typename T>
__device__ __noinline__ void clos_row(const T* __restrict__ up, const T* __restrict__ cp, long long fs, int Ss,
                                      T* __restrict__ r) {
    constexpr int NJ = CTab<O>::NJ;
    T uw[3][NJ];
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int c = 0; c < NJ; ++c) uw[l][c] = ldg(up + l * fs + (c - ROW) * Ss);
    T rr[3] = {T(0), T(0), T(0)};
    auto b = [&](int s6, int c) { return ldg(cp + s6 * fs + (c - ROW) * Ss); };
    clos_row_k<O, ROW>(uw, b, rr, std::make_integer_sequence<int, NJ>());
    r[0] += rr[0];
    r[1] += rr[1];
    r[2] += rr[2];
}

template <int O, typename T, int... R>
__device__ __forceinline__ void clos_dispatch(int row, const T* up, const T* cp, long long fs, int Ss, T* r,
                                              std::integer_sequence<int, R...>) {
    ((row == R ? clos_row<O, R>(up, cp, fs, Ss, r) : void()), ...);
}

// h^2 D_xx^FC rows of the closure (i < NCLOS or i >= N - NCLOS) for the node at index i of a line
// with stride S
template <int O, typename T>
__device__ __forceinline__ void dxx3_closure_ptr(int N, int i, const T* up, const T* cp, long long fs, int S,
                                                 T r[3]) {
    using P = Ord<O>;
    const bool right = i >= N - P::NCLOS;
    const int row = right ? N - 1 - i : i;
    clos_dispatch<O, T>(row, up, cp, fs, right ? -S : S, r, std::make_integer_sequence<int, P::NCLOS>());
}

template <int O, typename T, class FU, class FB>
__device__ __forceinline__ void dxx3_interior(int i, FU u, FB b, T r[3]) {
    constexpr int Q = Ord<O>::Q;
    T dp[3][Q], dm[3][Q];
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        const T uc = u(l, i);
#pragma unroll
        for (int m = 1; m <= Q; ++m) {
            dp[l][m - 1] = u(l, i + m) - uc;
            dm[l][m - 1] = u(l, i - m) - uc;
        }
    }
#pragma unroll
    for (int k = -Q; k <= Q; ++k) {
        T L[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int m = 1; m <= Q; ++m) {
            const T cp = edge_wT<O, T>(m, k), cn = edge_wT<O, T>(m, k + m);
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                if (cp != T(0)) L[l] += cp * dp[l][m - 1];
                if (cn != T(0)) L[l] += cn * dm[l][m - 1];
            }
        }
        const T b00 = b(0, i + k), b01 = b(1, i + k), b02 = b(2, i + k), b11 = b(3, i + k), b12 = b(4, i + k),
                b22 = b(5, i + k);
        r[0] += b00 * L[0] + b01 * L[1] + b02 * L[2];
        r[1] += b01 * L[0] + b11 * L[1] + b12 * L[2];
        r[2] += b02 * L[0] + b12 * L[1] + b22 * L[2];
    }
}

constexpr int BX = 32, BY = 8;

// element stride of direction D as a 32-bit int (a plane of the grid holds fewer than 2^31
// elements, checked at create): 1 along x1 (a compile-time constant), pitch or plane otherwise.
// Neighbour reads go through the node's own pointer plus (t - i) * stride, so interior stencil
// offsets fold into constants shared by every field.
template <int D> __device__ __forceinline__ int dstride(const Grid3& g) {
    if constexpr (D == 0) return 1;
    else return (int)g.s[D];
}

// D_D u_l (l = 0..2) at the node (index i along D), u at the node's pointer
template <typename T, int O, int D>
__device__ __forceinline__ void grad_dir(const Grid3& g, int i, const T* __restrict__ up, T gr[3]) {
    const int S = dstride<D>(g);
    const int N = g.n[D];
    const T ih = T(g.ih[D]);
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        const T* p = up + l * g.fs;
        gr[l] = ih * dsum<O, T>(N, i, [&](int t) { return ldg(p + (t - i) * S); });
    }
}

template <typename T, int NV> __device__ __forceinline__ void vld(const T* p, T v[NV]) {
    if constexpr (NV == 2 && sizeof(T) == 4) {
        const float2 x = __ldg(reinterpret_cast<const float2*>(p));
        v[0] = x.x;
        v[1] = x.y;
    } else {
#pragma unroll
        for (int n = 0; n < NV; ++n) v[n] = __ldg(p + n);
    }
}
template <typename T, int NV> __device__ __forceinline__ void vst(T* p, const T v[NV]) {
    if constexpr (NV == 2 && sizeof(T) == 4) {
        *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
    } else {
#pragma unroll
        for (int n = 0; n < NV; ++n) p[n] = v[n];
    }
}

// D_D u_l of one node as a call of its own (the closure rows of the paired flux kernel)
template <typename T, int O, int D>
__device__ __noinline__ void grad_call(const Grid3& g, int i, const T* __restrict__ up, T* __restrict__ out) {
    T gr[3];
    grad_dir<T, O, D>(g, i, up, gr);
    out[0] = gr[0];
    out[1] = gr[1];
    out[2] = gr[2];
}

// ------------------------------------------------------------------ mixed fluxes
// Two x1-adjacent nodes per thread (FP32; one node in FP64).  A pair whose x1 rows are interior
// reads its x1 stencil as aligned vector windows; its x2 / x3 rows are vector loads at +-k
// strides (interior) or the general rows node by node (closure rows, the same for a whole warp).
// A pair near the x1 faces takes the general rows for everything.
template <typename T, int O, int NV>
__device__ __forceinline__ void flux_pair(const Grid3& g, int i1, int i2, int i3, const T* __restrict__ up,
                                          T gr[NV][3][3]) {
    using P = Ord<O>;
    constexpr int Q = P::Q;
    constexpr int QA = (Q + NV - 1) / NV * NV;
    constexpr int WN = NV + 2 * QA;
    const long long fs = g.fs;
    const bool x1int = i1 >= P::NB && i1 + NV - 1 <= g.n[0] - 1 - P::NB && i1 >= QA;
    if (x1int) {
        const T ih = T(g.ih[0]);
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            T w[WN];
#pragma unroll
            for (int v = 0; v < WN / NV; ++v) vld<T, NV>(up + l * fs - QA + v * NV, w + v * NV);
#pragma unroll
            for (int n = 0; n < NV; ++n) {
                T acc = T(0);
#pragma unroll
                for (int k = 1; k <= Q; ++k) acc += P::template aT<T>(k - 1) * (w[QA + n + k] - w[QA + n - k]);
                gr[n][0][l] = ih * acc;
            }
        }
    } else {
#pragma unroll
        for (int n = 0; n < NV; ++n) grad_call<T, O, 0>(g, i1 + n, up + n, gr[n][0]);
    }
    auto strided = [&](auto dc, int i) {
        constexpr int D = decltype(dc)::value;
        const int N = g.n[D];
        if (i >= P::NB && i <= N - 1 - P::NB) {
            const int S = dstride<D>(g);
            const T ih = T(g.ih[D]);
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                T acc[NV];
#pragma unroll
                for (int n = 0; n < NV; ++n) acc[n] = T(0);
#pragma unroll
                for (int k = 1; k <= Q; ++k) {
                    T a[NV], b[NV];
                    vld<T, NV>(up + l * fs + k * S, a);
                    vld<T, NV>(up + l * fs - k * S, b);
                    const T ak = P::template aT<T>(k - 1);
#pragma unroll
                    for (int n = 0; n < NV; ++n) acc[n] += ak * (a[n] - b[n]);
                }
#pragma unroll
                for (int n = 0; n < NV; ++n) gr[n][D][l] = ih * acc[n];
            }
        } else {
#pragma unroll
            for (int n = 0; n < NV; ++n) grad_call<T, O, D>(g, i, up + n, gr[n][D]);
        }
    };
    strided(std::integral_constant<int, 1>(), i2);
    strided(std::integral_constant<int, 2>(), i3);
}

template <typename T, int O, int NV>
__global__ void __launch_bounds__(BX * BY, 3) k3_flux(Grid3 g, const T* __restrict__ u, const T* __restrict__ cm,
                                                   T* __restrict__ q) {
    const int i1 = (blockIdx.x * BX + threadIdx.x) * NV, i2 = blockIdx.y * BY + threadIdx.y, i3 = blockIdx.z;
    if (i1 >= g.n[0] || i2 >= g.n[1]) return;
    const long long o = i1 + i2 * g.s[1] + i3 * g.s[2];
    const long long fs = g.fs;
    const T* up = u + o;
    // the last pair of an odd row has one node: it runs alone through the general rows
    const bool full = i1 + NV - 1 < g.n[0];
    T gr[NV][3][3];                               // gr[n][k][l] = D_k u_l at node n
    if (full) {
        flux_pair<T, O, NV>(g, i1, i2, i3, up, gr);
    } else {
#pragma unroll
        for (int n = 0; n < NV; ++n) {
            grad_call<T, O, 0>(g, i1, up, gr[n][0]);
            grad_call<T, O, 1>(g, i2, up, gr[n][1]);
            grad_call<T, O, 2>(g, i3, up, gr[n][2]);
        }
    }
    T qq[NV][3][3];
#pragma unroll
    for (int n = 0; n < NV; ++n)
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) qq[n][i][j] = T(0);
    const T* cmo = cm + o;
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const int i = p == 2 ? 1 : 0, k = p == 0 ? 1 : 2;
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                T M[NV];
                if (full) {
                    vld<T, NV>(cmo + (9 * p + 3 * j + l) * fs, M);
                } else {
                    M[0] = ldg(cmo + (9 * p + 3 * j + l) * fs);
#pragma unroll
                    for (int n = 1; n < NV; ++n) M[n] = T(0);
                }
#pragma unroll
                for (int n = 0; n < NV; ++n) {
                    qq[n][i][j] += M[n] * gr[n][k][l];       // c_ijkl D_k u_l
                    qq[n][k][l] += M[n] * gr[n][i][j];       // c_klij D_i u_j (major symmetry)
                }
            }
    }
    T* qo = q + o;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const long long f = (3 * i + j) * fs;
            if (full) {
                T v[NV];
#pragma unroll
                for (int n = 0; n < NV; ++n) v[n] = qq[n][i][j];
                vst<T, NV>(qo + f, v);
            } else {
                qo[f] = qq[0][i][j];
            }
        }
}

// ------------------------------------------------------------------ divergence and leapfrog store
// r_j += D_D q_Dj + D_DD^FC(c_DjDl) u_l for one direction D
// x1 closure rows as matrices: row rho of the line (i2, i3) at side s is
//   h^2 D_xx^FC(b) u |_rho = sum_c sum_l M_{s,rho,c}(b_jl) u_l(col_s(c)),  M(b) = sum_{t in row: j_t = c} c_t b(k_t)
// (symmetric in jl like b), formed once from the material by k3_xclos.  Layout
// xm[(((s * NJ + c) * 6 + s6) * nlines + line) * NCLOS + rho]: the row index is fastest, so the lanes
// of a warp (consecutive i1, hence consecutive rows) read consecutive words, and every lane runs
// the same code whatever its row.
struct XClos {
    const void* m;
    long long nlines;
};

template <typename T, int O>
__device__ __forceinline__ void xclos_apply(const XClos& xc, int N, int i, int line, const T* __restrict__ up,
                                            long long fs, T rr[3]) {
    using P = Ord<O>;
    constexpr int NJ = CTab<O>::NJ, NC = P::NCLOS;
    const bool right = i >= N - NC;
    const int rho = right ? N - 1 - i : i;
    const T* mp = static_cast<const T*>(xc.m) + ((long long)(right ? NJ : 0) * 6 * xc.nlines + line) * NC + rho;
    const long long cs = xc.nlines * NC;            // stride of one (c, s6) slot
#pragma unroll
    for (int c = 0; c < NJ; ++c) {
        const int off = right ? (N - 1 - c) - i : c - i;
        const T u0 = ldg(up + off), u1 = ldg(up + fs + off), u2 = ldg(up + 2 * fs + off);
        T m6[6];
#pragma unroll
        for (int s6 = 0; s6 < 6; ++s6) m6[s6] = ldg(mp + (long long)(c * 6 + s6) * cs);
        rr[0] += m6[0] * u0 + m6[1] * u1 + m6[2] * u2;
        rr[1] += m6[1] * u0 + m6[3] * u1 + m6[4] * u2;
        rr[2] += m6[2] * u0 + m6[4] * u1 + m6[5] * u2;
    }
}

template <typename T, int O, int D>
__device__ __forceinline__ void div_dir(const Grid3& g, int i, const T* __restrict__ qo, const T* __restrict__ cdo,
                                        const T* __restrict__ up, T r[3], const XClos* xc = nullptr, int line = 0) {
    const int S = dstride<D>(g);
    const int N = g.n[D];
    const long long fs = g.fs;
    const T ih = T(g.ih[D]);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const T* p = qo + (3 * D + j) * fs;
        r[j] += ih * dsum<O, T>(N, i, [&](int t) { return ldg(p + (t - i) * S); });
    }
    T rr[3] = {T(0), T(0), T(0)};
    const T* cp = cdo + 6 * D * fs;
    if (i < Ord<O>::NCLOS || i >= N - Ord<O>::NCLOS) {
        if constexpr (D == 0) xclos_apply<T, O>(*xc, N, i, line, up, fs, rr);
        else dxx3_closure_ptr<O, T>(N, i, up, cp, fs, S, rr);
    } else {
        dxx3_interior<O, T>(i, [&](int l, int t) { return ldg(up + l * fs + (t - i) * S); },
                            [&](int s, int t) { return ldg(cp + s * fs + (t - i) * S); }, rr);
    }
    const T ih2 = ih * ih;
#pragma unroll
    for (int j = 0; j < 3; ++j) r[j] += ih2 * rr[j];
}

// the x1 closure matrices of the lines of x3-planes k0 <= i3 < k0 + nk (one thread per line, side, row)
template <typename T, int O>
__global__ void __launch_bounds__(128) k3_xclos(Grid3 g, int k0, int nk, const T* __restrict__ cd, T* __restrict__ xm) {
    using P = Ord<O>;
    constexpr int NJ = CTab<O>::NJ, NC = P::NCLOS;
    const int i2 = blockIdx.x * blockDim.x + threadIdx.x;
    const int i3 = k0 + blockIdx.y;
    const int rho = blockIdx.z % NC, side = blockIdx.z / NC;
    if (i2 >= g.n[1] || blockIdx.y >= (unsigned)nk) return;
    const int N = g.n[0];
    const long long nlines = (long long)g.n[1] * g.n[2];
    const long long line = (long long)i3 * g.n[1] + i2;
    const long long base = i2 * g.s[1] + i3 * g.s[2];
    for (int c = 0; c < NJ; ++c)
        for (int s6 = 0; s6 < 6; ++s6) {
            double m = 0.0;
            for (int t = P::cstart(rho); t < P::cstart(rho + 1); ++t) {
                if (P::cj(t) != c) continue;
                const int k = side ? N - 1 - P::ck(t) : P::ck(t);
                m += P::cc(t) * double(cd[s6 * g.fs + base + k]);
            }
            xm[((((long long)side * NJ + c) * 6 + s6) * nlines + line) * NC + rho] = T(m);
        }
}

// ------------------------------------------------------------------ divergence: interior box and boundary shell
// Nodes at least max(NCLOS, NCOL) from the x1 faces use interior rows along x1 and no x1-face
// SAT.  They form the box [x1lo, x1hi) x [y0, y1) x [z0, z1) (x1lo a multiple of NV; the box
// spans every i2 and i3), handled by k3_div_int: NV consecutive x1 nodes per thread read as one
// vector (float2 for FP32); the x2 and x3 rows are interior vector code or, on the closure planes
// and rows (the same for the whole warp), the general rows.  The x1 slabs outside the box (the
// shell) go to k3_div_shell.
struct Box3 {
    int x1lo, x1hi, y0, y1, z0, z1;
};

// x2 / x3 direction (stride S) for NV nodes: r[n][j] += ih D q_Dj + ih^2 D_xx(b) u, interior rows
template <typename T, int O, int NV>
__device__ __forceinline__ void div_int_strided(const T* __restrict__ qD, const T* __restrict__ cdD,
                                                const T* __restrict__ up, long long fs, int S, T ih, T r[NV][3]) {
    constexpr int Q = Ord<O>::Q;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        T acc[NV];
#pragma unroll
        for (int n = 0; n < NV; ++n) acc[n] = T(0);
        const T* p = qD + j * fs;
#pragma unroll
        for (int k = 1; k <= Q; ++k) {
            T a[NV], b[NV];
            vld<T, NV>(p + k * S, a);
            vld<T, NV>(p - k * S, b);
            const T ak = Ord<O>::template aT<T>(k - 1);
#pragma unroll
            for (int n = 0; n < NV; ++n) acc[n] += ak * (a[n] - b[n]);
        }
#pragma unroll
        for (int n = 0; n < NV; ++n) r[n][j] += ih * acc[n];
    }
    T dp[3][Q][NV], dm[3][Q][NV];
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        T uc[NV];
        vld<T, NV>(up + l * fs, uc);
#pragma unroll
        for (int m = 1; m <= Q; ++m) {
            T a[NV], b[NV];
            vld<T, NV>(up + l * fs + m * S, a);
            vld<T, NV>(up + l * fs - m * S, b);
#pragma unroll
            for (int n = 0; n < NV; ++n) {
                dp[l][m - 1][n] = a[n] - uc[n];
                dm[l][m - 1][n] = b[n] - uc[n];
            }
        }
    }
    const T ih2 = ih * ih;
#pragma unroll
    for (int k = -Q; k <= Q; ++k) {
        T L[3][NV];
#pragma unroll
        for (int l = 0; l < 3; ++l)
#pragma unroll
            for (int n = 0; n < NV; ++n) L[l][n] = T(0);
#pragma unroll
        for (int m = 1; m <= Q; ++m) {
            const T cp = edge_wT<O, T>(m, k), cn = edge_wT<O, T>(m, k + m);
#pragma unroll
            for (int l = 0; l < 3; ++l)
#pragma unroll
                for (int n = 0; n < NV; ++n) {
                    if (cp != T(0)) L[l][n] += cp * dp[l][m - 1][n];
                    if (cn != T(0)) L[l][n] += cn * dm[l][m - 1][n];
                }
        }
        T bb[6][NV];
#pragma unroll
        for (int s6 = 0; s6 < 6; ++s6) vld<T, NV>(cdD + s6 * fs + k * S, bb[s6]);
#pragma unroll
        for (int n = 0; n < NV; ++n) {
            r[n][0] += ih2 * (bb[0][n] * L[0][n] + bb[1][n] * L[1][n] + bb[2][n] * L[2][n]);
            r[n][1] += ih2 * (bb[1][n] * L[0][n] + bb[3][n] * L[1][n] + bb[4][n] * L[2][n]);
            r[n][2] += ih2 * (bb[2][n] * L[0][n] + bb[4][n] * L[1][n] + bb[5][n] * L[2][n]);
        }
    }
}

// the same for FP32 node pairs, in packed FP32x2 arithmetic (one instruction for both nodes)
__device__ __forceinline__ float2 p2ffma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p2fmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p2fsub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 p2s(float a) { return make_float2(a, a); }

template <int O>
__device__ __forceinline__ void div_int_strided_f2(const float* __restrict__ qD, const float* __restrict__ cdD,
                                                   const float* __restrict__ up, long long fs, int S, float ih,
                                                   float r[2][3]) {
    constexpr int Q = Ord<O>::Q;
    auto ld2 = [](const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); };
    float2 R[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float* p = qD + j * fs;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 1; k <= Q; ++k)
            acc = p2ffma(p2s(Ord<O>::template aT<float>(k - 1)), p2fsub(ld2(p + k * S), ld2(p - k * S)), acc);
        R[j] = p2fmul(p2s(ih), acc);
    }
    float2 dp[3][Q], dm[3][Q];
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        const float2 uc = ld2(up + l * fs);
#pragma unroll
        for (int m = 1; m <= Q; ++m) {
            dp[l][m - 1] = p2fsub(ld2(up + l * fs + m * S), uc);
            dm[l][m - 1] = p2fsub(ld2(up + l * fs - m * S), uc);
        }
    }
    const float2 ih2 = p2s(ih * ih);
#pragma unroll
    for (int k = -Q; k <= Q; ++k) {
        float2 L[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
        for (int m = 1; m <= Q; ++m) {
            const float cp = edge_wT<O, float>(m, k), cn = edge_wT<O, float>(m, k + m);
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                if (cp != 0.f) L[l] = p2ffma(p2s(cp), dp[l][m - 1], L[l]);
                if (cn != 0.f) L[l] = p2ffma(p2s(cn), dm[l][m - 1], L[l]);
            }
        }
        float2 bb[6];
#pragma unroll
        for (int s6 = 0; s6 < 6; ++s6) bb[s6] = ld2(cdD + s6 * fs + k * S);
        const float2 t0 = p2ffma(bb[2], L[2], p2ffma(bb[1], L[1], p2fmul(bb[0], L[0])));
        const float2 t1 = p2ffma(bb[4], L[2], p2ffma(bb[3], L[1], p2fmul(bb[1], L[0])));
        const float2 t2 = p2ffma(bb[5], L[2], p2ffma(bb[4], L[1], p2fmul(bb[2], L[0])));
        R[0] = p2ffma(ih2, t0, R[0]);
        R[1] = p2ffma(ih2, t1, R[1]);
        R[2] = p2ffma(ih2, t2, R[2]);
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        r[0][j] += R[j].x;
        r[1][j] += R[j].y;
    }
}

// x1 direction for NV consecutive nodes: windows of WN = NV + 2 QA values from i1 - QA (QA = Q
// rounded up to NV, so the window loads stay vector-aligned); node n sits at window index QA + n
template <typename T, int O, int NV>
__device__ __forceinline__ void div_int_x1(const T* __restrict__ q0, const T* __restrict__ cd0,
                                           const T* __restrict__ up, long long fs, T ih, T r[NV][3]) {
    constexpr int Q = Ord<O>::Q;
    constexpr int QA = (Q + NV - 1) / NV * NV;
    constexpr int WN = NV + 2 * QA;
    auto window = [&](const T* p, T w[WN]) {
#pragma unroll
        for (int v = 0; v < WN / NV; ++v) vld<T, NV>(p - QA + v * NV, w + v * NV);
    };
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        T w[WN];
        window(q0 + j * fs, w);
#pragma unroll
        for (int n = 0; n < NV; ++n) {
            T acc = T(0);
#pragma unroll
            for (int k = 1; k <= Q; ++k) acc += Ord<O>::template aT<T>(k - 1) * (w[QA + n + k] - w[QA + n - k]);
            r[n][j] += ih * acc;
        }
    }
    // narrow rows one displacement component at a time (L_k of u_l for the NV nodes, then every
    // coefficient field b_jl that multiplies u_l), so only one component's L's are live
    const T ih2 = ih * ih;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        T L[2 * Q + 1][NV];
        {
            T w[WN];
            window(up + l * fs, w);
#pragma unroll
            for (int n = 0; n < NV; ++n) {
                const T uc = w[QA + n];
#pragma unroll
                for (int k = -Q; k <= Q; ++k) {
                    T acc = T(0);
#pragma unroll
                    for (int m = 1; m <= Q; ++m) {
                        const T cp = edge_wT<O, T>(m, k), cn = edge_wT<O, T>(m, k + m);
                        if (cp != T(0)) acc += cp * (w[QA + n + m] - uc);
                        if (cn != T(0)) acc += cn * (w[QA + n - m] - uc);
                    }
                    L[k + Q][n] = acc;
                }
            }
        }
        // fields b_jl with this l: (j, l) for j = 0..2, s6 = sym3 index
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int s6 = j <= l ? (j == 0 ? l : (j == 1 ? 2 + l : 5)) : (l == 0 ? j : (l == 1 ? 2 + j : 5));
            T w[WN];
            window(cd0 + s6 * fs, w);
#pragma unroll
            for (int n = 0; n < NV; ++n) {
                T acc = T(0);
#pragma unroll
                for (int k = -Q; k <= Q; ++k) acc += w[QA + n + k] * L[k + Q][n];
                r[n][j] += ih2 * acc;
            }
        }
    }
}

// ------------------------------------------------------------------ boundary SATs of the faces x_m = 0, 1
// Computed by the shell kernel for the nodes they reach, so no node is written twice:
//   traction:     J SAT_J = -H^-1 P_f nu c_mJkL D_k u_L              (face node only)
//   displacement: J SAT_J = H^-1 [ sum_k D_k^T (nu c_mLkJ P_f u_L) - P_f (beta d / h1) c_mJmL u_L ]
// H^-1 P_f is 1 / (h_m hw_0) at a face node; D_m^T spreads the normal term over the first NCOL
// nodes of the normal line (H^-1 D_m^T at depth t: D_m[face][t] / (h_m hw_t)); the tangential
// D_k^T stays on the face, weighted by hw_k(a') / hw_k(a).
// tangential transpose along direction K of face direction M: (H_K^-1 D_K^T H_K v)(a) with
// v_J = nu c_MLKJ u_L on the face; away from the ends of the line (every row that reads column a
// is an interior row and every weight there is 1) this is -(D_K v)(a).
template <typename T, int O, int M, int K>
__device__ __forceinline__ void face_tangential(const Grid3& g, int ak, const T* __restrict__ up,
                                               const T* __restrict__ cm, const T* __restrict__ cd, long long o,
                                               T base, T rs[3]) {
    using P = Ord<O>;
    const int Nk = g.n[K];
    const int S = dstride<K>(g);
    const long long fs = g.fs;
    auto vJ = [&](int off, T out[3]) {
        T v[3];
#pragma unroll
        for (int L = 0; L < 3; ++L) v[L] = ldg(up + L * fs + off);
#pragma unroll
        for (int J = 0; J < 3; ++J) {
            T s = T(0);
#pragma unroll
            for (int L = 0; L < 3; ++L) s += cfull(cm, cd, fs, M, L, K, J, o + off) * v[L];
            out[J] = s;
        }
    };
    if (ak >= P::NCOL && ak >= P::NB + P::Q && ak <= Nk - 1 - P::NCOL && ak <= Nk - 1 - P::NB - P::Q) {
#pragma unroll
        for (int mm = 1; mm <= P::Q; ++mm) {
            const T am = P::template aT<T>(mm - 1) * base;
            T vp[3], vm[3];
            vJ(mm * S, vp);
            vJ(-mm * S, vm);
#pragma unroll
            for (int J = 0; J < 3; ++J) rs[J] += am * (vm[J] - vp[J]);
        }
    } else {
        constexpr int W = P::NCOL - 1 > P::Q ? P::NCOL - 1 : P::Q;
        const int lo = ak - W < 0 ? 0 : ak - W, hi = ak + W > Nk - 1 ? Nk - 1 : ak + W;
        const T iwa = T(1.0 / hweight<O>(Nk, ak));
        for (int a2 = lo; a2 <= hi; ++a2) {
            const T dc = dcoefT<O, T>(Nk, a2, ak);
            if (dc == T(0)) continue;
            const T coef = base * dc * hweightT<O, T>(Nk, a2) * iwa;
            T v[3];
            vJ((a2 - ak) * S, v);
#pragma unroll
            for (int J = 0; J < 3; ++J) rs[J] += coef * v[J];
        }
    }
}

struct Faces3 {
    int kind[6];            // BC_DISPLACEMENT or BC_TRACTION per face
    double beta;
};

// r += the SAT terms of the faces x_M = 0 and x_M = 1 that reach the node (index im along M):
// at a face node the face's own terms, at depth 1 .. NCOL-1 below a displacement face the
// normal transpose D_M^T of that face's node on the same line.
template <typename T, int O, int M>
__device__ __noinline__ void face_terms(const Grid3& g, const Faces3& fc, int im, int ia, int ib, long long o,
                                           const T* __restrict__ u, const T* __restrict__ cm,
                                           const T* __restrict__ cd, T r[3]) {
    using P = Ord<O>;
    constexpr int PD = M == 0 ? 1 : 0, TD = M == 2 ? 1 : 2;
    const int Nm = g.n[M];
    const int SM = dstride<M>(g);
    const long long fs = g.fs;
    const T ihm = T(g.ih[M]);
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const int depth = side ? Nm - 1 - im : im;
        if (depth >= P::NCOL) continue;
        const int kind = fc.kind[2 * M + side];
        const T nu = side ? T(1) : T(-1);
        const int frow = side ? Nm - 1 : 0;                 // the face's row along M
        if (depth > 0) {
            if (kind != BC_DISPLACEMENT) continue;
            const T dc = dcoefT<O, T>(Nm, frow, im);
            if (dc == T(0)) continue;
            const long long of = o + (long long)(frow - im) * SM;
            T uf[3];
#pragma unroll
            for (int L = 0; L < 3; ++L) uf[L] = ldg(u + L * fs + of);
            const T coef = ihm * ihm * dc / hweightT<O, T>(Nm, im) * nu;
#pragma unroll
            for (int J = 0; J < 3; ++J) {
                T sm = T(0);
#pragma unroll
                for (int L = 0; L < 3; ++L) sm += cfull(cm, cd, fs, M, L, M, J, of) * uf[L];
                r[J] += coef * sm;
            }
            continue;
        }
        const T* up = u + o;
        const T ihb = ihm / hweightT<O, T>(Nm, im);         // H^-1 P_f at the face node
        if (kind == BC_TRACTION) {
            T gr[3][3];
            const int ix[3] = {M == 0 ? im : ia, M == 1 ? im : (M == 0 ? ia : ib), M == 2 ? im : ib};
            grad_dir<T, O, 0>(g, ix[0], up, gr[0]);
            grad_dir<T, O, 1>(g, ix[1], up, gr[1]);
            grad_dir<T, O, 2>(g, ix[2], up, gr[2]);
#pragma unroll
            for (int J = 0; J < 3; ++J) {
                T sm = T(0);
#pragma unroll
                for (int k = 0; k < 3; ++k)
#pragma unroll
                    for (int L = 0; L < 3; ++L) sm += cfull(cm, cd, fs, M, J, k, L, o) * gr[k][L];
                r[J] -= ihb * nu * sm;
            }
        } else {
            T uf[3];
#pragma unroll
            for (int L = 0; L < 3; ++L) uf[L] = ldg(up + L * fs);
            // penalty -H^-1 P_f (beta d / h1) c_mJmL u_L (h1 = h_m hw_0), and the normal transpose at
            // depth 0, H^-1 D_M[face][face] nu c_MLMJ u_L
            const T pen = T(fc.beta * 3.0) * ihb * ihb;
            const T cn = ihm * ihm * dcoefT<O, T>(Nm, frow, im) / hweightT<O, T>(Nm, im) * nu;
#pragma unroll
            for (int J = 0; J < 3; ++J) {
                T sp = T(0), sn = T(0);
#pragma unroll
                for (int L = 0; L < 3; ++L) {
                    sp += cfull(cm, cd, fs, M, J, M, L, o) * uf[L];
                    sn += cfull(cm, cd, fs, M, L, M, J, o) * uf[L];
                }
                r[J] += cn * sn - pen * sp;
            }
            const T base = ihb * nu;
            face_tangential<T, O, M, PD>(g, ia, up, cm, cd, o, base * T(g.ih[PD]), r);
            face_tangential<T, O, M, TD>(g, ib, up, cm, cd, o, base * T(g.ih[TD]), r);
        }
    }
}

// the general row code of one node as a call of its own, so the closure planes do not weigh on
// the register allocation of the vector path
template <typename T, int O, int D>
__device__ __noinline__ void div_dir_call(const Grid3& g, int i, const T* __restrict__ qo, const T* __restrict__ cdo,
                                          const T* __restrict__ up, T* __restrict__ rn) {
    T r3[3] = {T(0), T(0), T(0)};
    div_dir<T, O, D>(g, i, qo, cdo, up, r3);
    rn[0] += r3[0];
    rn[1] += r3[1];
    rn[2] += r3[2];
}

// direction D = x2 or x3 for the NV nodes of a thread: interior rows through the vector code,
// closure rows (the same for every lane of a warp, whose lanes share i2 and i3) node by node
template <typename T, int O, int NV, int D>
__device__ __forceinline__ void div_int_dir(const Grid3& g, int i, const T* __restrict__ qo,
                                            const T* __restrict__ cdo, const T* __restrict__ up, T r[NV][3]) {
    const int N = g.n[D];
    const long long fs = g.fs;
    if (i >= Ord<O>::NCLOS && i < N - Ord<O>::NCLOS) {
        if constexpr (NV == 2 && sizeof(T) == 4)
            div_int_strided_f2<O>(qo + 3 * D * fs, cdo + 6 * D * fs, up, fs, dstride<D>(g), float(g.ih[D]), r);
        else
            div_int_strided<T, O, NV>(qo + 3 * D * fs, cdo + 6 * D * fs, up, fs, dstride<D>(g), T(g.ih[D]), r);
        return;
    }
#pragma unroll
    for (int n = 0; n < NV; ++n) div_dir_call<T, O, D>(g, i, qo + n, cdo + n, up + n, r[n]);
}

// MODE 0: leapfrog in increment form, d = du + dt^2 w r, un = u + d (du updated in place);
// MODE 1: apply, out = w r.
// launch shapes of k3_div_int (sbp3_set_tuning / sbp3_autotune): x2 rows per block and the
// minimum resident blocks per SM, which sets the register cap (65536 / (32 BY MINB))
struct DivShape {
    int by, minb;
};
constexpr DivShape kDivShapes[4] = {{4, 5}, {4, 6}, {8, 3}, {2, 10}};

template <typename T, int O, int MODE, int NV, int BY, int MINB>
__global__ void __launch_bounds__(32 * BY, MINB) k3_div_int(Grid3 g, Box3 bx, Faces3 fc, const T* __restrict__ u,
                                                            const T* __restrict__ q, const T* __restrict__ cm,
                                                            const T* __restrict__ cd, const T* __restrict__ w,
                                                            T* __restrict__ du, T* __restrict__ un, T dt2) {
    using P = Ord<O>;
    const int gx = blockIdx.x * 32 + threadIdx.x;
    const int i1 = bx.x1lo + gx * NV, i2 = bx.y0 + blockIdx.y * BY + threadIdx.y, i3 = bx.z0 + blockIdx.z;
    if (i1 >= bx.x1hi || i2 >= bx.y1) return;
    const long long o = i1 + i2 * g.s[1] + i3 * g.s[2];
    const long long fs = g.fs;
    const T* up = u + o;
    T r[NV][3];
#pragma unroll
    for (int n = 0; n < NV; ++n) r[n][0] = r[n][1] = r[n][2] = T(0);
    div_int_x1<T, O, NV>(q + o, cd + o, up, fs, T(g.ih[0]), r);
    div_int_dir<T, O, NV, 1>(g, i2, q + o, cd + o, up, r);
    div_int_dir<T, O, NV, 2>(g, i3, q + o, cd + o, up, r);
    // SATs of the x2 and x3 faces that reach these nodes (the x1 faces lie in the shell)
    if (i2 < P::NCOL || i2 >= g.n[1] - P::NCOL) {
#pragma unroll
        for (int n = 0; n < NV; ++n) face_terms<T, O, 1>(g, fc, i2, i1 + n, i3, o + n, u, cm, cd, r[n]);
    }
    if (i3 < P::NCOL || i3 >= g.n[2] - P::NCOL) {
#pragma unroll
        for (int n = 0; n < NV; ++n) face_terms<T, O, 2>(g, fc, i3, i1 + n, i2, o + n, u, cm, cd, r[n]);
    }
    T wv[NV];
    vld<T, NV>(w + o, wv);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const long long oj = j * fs + o;
        T out[NV];
        if constexpr (MODE == 0) {
            T d[NV], uc[NV];
            vld<T, NV>(du + oj, d);
            vld<T, NV>(up + j * fs, uc);
#pragma unroll
            for (int n = 0; n < NV; ++n) {
                d[n] += dt2 * wv[n] * r[n][j];
                out[n] = uc[n] + d[n];
            }
            vst<T, NV>(du + oj, d);
        } else {
#pragma unroll
            for (int n = 0; n < NV; ++n) out[n] = wv[n] * r[n][j];
        }
        vst<T, NV>(un + oj, out);
    }
}

// the shell: every node outside the box, lanes along x1 (coalesced), in three parts:
//   Z: the planes i3 < z0, i3 >= z1 (whole planes);
//   Y: within the box's planes, the rows i2 < y0, i2 >= y1 (whole rows);
//   X: within the box's planes and rows, the x1 runs i1 < x1lo and i1 >= x1hi.
struct Shell3 {
    long long cZ, cY, cX;   // node counts of the three parts
};

__device__ __forceinline__ bool shell_node(const Grid3& g, const Box3& bx, const Shell3& sh, long long t, int& i1,
                                           int& i2, int& i3) {
    const long long n1 = g.n[0], n2 = g.n[1];
    const long long plane = n1 * n2;
    if (t < sh.cZ) {
        const long long pz = t / plane;
        const long long rem = t - pz * plane;
        i3 = (int)(pz < bx.z0 ? pz : bx.z1 + (pz - bx.z0));
        i2 = (int)(rem / n1);
        i1 = (int)(rem - (long long)i2 * n1);
        return true;
    }
    t -= sh.cZ;
    if (t < sh.cY) {
        const long long rowsB = bx.y0 + (n2 - bx.y1);
        const long long row = t / n1;
        i1 = (int)(t - row * n1);
        const long long pz = row / rowsB, ry = row - pz * rowsB;
        i3 = (int)(bx.z0 + pz);
        i2 = (int)(ry < bx.y0 ? ry : bx.y1 + (ry - bx.y0));
        return true;
    }
    t -= sh.cY;
    if (t >= sh.cX) return false;
    const long long ny = bx.y1 - bx.y0;
    const long long runs = bx.x1lo + (n1 - bx.x1hi);
    const long long row = t / runs, rx = t - row * runs;
    const long long pz = row / ny, py = row - pz * ny;
    i3 = (int)(bx.z0 + pz);
    i2 = (int)(bx.y0 + py);
    i1 = (int)(rx < bx.x1lo ? rx : bx.x1hi + (rx - bx.x1lo));
    return true;
}

// the boundary shell: volume terms with closure rows, then every face SAT reaching the node, then
// the leapfrog store (MODE as in k3_div_int)
template <typename T, int O, int MODE>
__global__ void __launch_bounds__(128) k3_div_shell(Grid3 g, Box3 bx, Shell3 sh, XClos xc, Faces3 fc, long long count,
                                                    const T* __restrict__ u, const T* __restrict__ q,
                                                    const T* __restrict__ cm, const T* __restrict__ cd,
                                                    const T* __restrict__ w, T* __restrict__ du,
                                                    T* __restrict__ un, T dt2) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    int i1, i2, i3;
    if (!shell_node(g, bx, sh, t, i1, i2, i3)) return;
    const long long o = i1 + i2 * g.s[1] + i3 * g.s[2];
    const T* up = u + o;
    const T* qo = q + o;
    const T* cdo = cd + o;
    T r[3] = {T(0), T(0), T(0)};
    div_dir<T, O, 0>(g, i1, qo, cdo, up, r, &xc, i3 * g.n[1] + i2);
    div_dir<T, O, 1>(g, i2, qo, cdo, up, r);
    div_dir<T, O, 2>(g, i3, qo, cdo, up, r);
    face_terms<T, O, 0>(g, fc, i1, i2, i3, o, u, cm, cd, r);
    face_terms<T, O, 1>(g, fc, i2, i1, i3, o, u, cm, cd, r);
    face_terms<T, O, 2>(g, fc, i3, i1, i2, o, u, cm, cd, r);
    const T wv = ldg(w + o);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const long long oj = j * g.fs + o;
        if constexpr (MODE == 0) {
            const T d = du[oj] + dt2 * wv * r[j];
            du[oj] = d;
            un[oj] = ldg(up + j * g.fs) + d;
        } else {
            un[oj] = wv * r[j];
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
