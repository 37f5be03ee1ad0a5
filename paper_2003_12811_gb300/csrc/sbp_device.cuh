// Device-side SBP building blocks shared by the libsbp kernels: coefficient tables in constant
// memory, 1-D first-derivative rows, fully compatible narrow second-derivative rows, and the
// block / face views the kernels receive.  Sec. 4 (operators), 4.3-4.7 (multi-D operator).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace sbpdev {
#define SBP_TABLE static __constant__
#include "sbp_tables.inc"
#undef SBP_TABLE
}  // namespace sbpdev

namespace sbp {

// ------------------------------------------------------------------ order traits
template <int O> struct Ord;
// Every coefficient is also available in the arithmetic type T (FP32 kernels read the FP32 twin
// tables, which hold exactly the values a cast of the FP64 entries gives).
#define SBP_TWIN(name, expr64, expr32)                                                                 \
    template <typename T> static __device__ __forceinline__ T name {                                   \
        if constexpr (sizeof(T) == 4) return expr32; else return expr64;                               \
    }
#define SBP_ORD(O)                                                                                     \
    template <> struct Ord<O> {                                                                        \
        static constexpr int Q = SBP##O##_Q, NB = SBP##O##_NB, NCOL = SBP##O##_NCOL,                   \
                             NCLOS = SBP##O##_NCLOS, NCLOSJ = SBP##O##_NCLOSJ, GS = SBP##O##_GS;       \
        static __device__ __forceinline__ double hw(int i) { return sbpdev::sbp##O##_HW[i]; }          \
        static __device__ __forceinline__ double dq(int r, int c) { return sbpdev::sbp##O##_DQ[r][c]; } \
        static __device__ __forceinline__ double a(int k) { return sbpdev::sbp##O##_A[k]; }            \
        static __device__ __forceinline__ int cstart(int r) { return sbpdev::sbp##O##_CLOS_START[r]; }  \
        static __device__ __forceinline__ int cj(int t) { return sbpdev::sbp##O##_CLOS_J[t]; }          \
        static __device__ __forceinline__ int ck(int t) { return sbpdev::sbp##O##_CLOS_K[t]; }          \
        static __device__ __forceinline__ double cc(int t) { return sbpdev::sbp##O##_CLOS_C[t]; }      \
        SBP_TWIN(hwT(int i), sbpdev::sbp##O##_HW[i], sbpdev::sbp##O##_HW_F[i])                          \
        SBP_TWIN(dqT(int r, int c), sbpdev::sbp##O##_DQ[r][c], sbpdev::sbp##O##_DQ_F[r][c])             \
        SBP_TWIN(aT(int k), sbpdev::sbp##O##_A[k], sbpdev::sbp##O##_A_F[k])                             \
        SBP_TWIN(ccT(int t), sbpdev::sbp##O##_CLOS_C[t], sbpdev::sbp##O##_CLOS_C_F[t])                  \
        /* gradient tables: node k < GS from the left end */                                            \
        static __device__ __forceinline__ int gn_start(int k) { return sbpdev::sbp##O##_GN_START[k]; }  \
        static __device__ __forceinline__ int gn_row(int t) { return sbpdev::sbp##O##_GN_ROW[t]; }      \
        static __device__ __forceinline__ int gn_j(int t) { return sbpdev::sbp##O##_GN_J[t]; }          \
        SBP_TWIN(gn_c(int t), sbpdev::sbp##O##_GN_C[t], sbpdev::sbp##O##_GN_C_F[t])                     \
        static __device__ __forceinline__ int dt_start(int k) { return sbpdev::sbp##O##_DT_START[k]; }  \
        static __device__ __forceinline__ int dt_row(int t) { return sbpdev::sbp##O##_DT_ROW[t]; }      \
        SBP_TWIN(dt_c(int t), sbpdev::sbp##O##_DT_C[t], sbpdev::sbp##O##_DT_C_F[t])                     \
    };
SBP_ORD(2)
SBP_ORD(4)
SBP_ORD(6)
#undef SBP_ORD
#undef SBP_TWIN

// interior edge weights E_m(i) = sum_k e_{m,k} b_{i+k} (m = 1..Q) of the narrow operator
template <int O> struct Edge;
template <> struct Edge<2> {
    template <typename T, class F> __device__ static __forceinline__ T e(int m, F B) { return SBP2_E1(B); }
};
template <> struct Edge<4> {
    template <typename T, class F> __device__ static __forceinline__ T e(int m, F B) {
        return m == 1 ? SBP4_E1(B) : SBP4_E2(B);
    }
};
template <> struct Edge<6> {
    template <typename T, class F> __device__ static __forceinline__ T e(int m, F B) {
        return m == 1 ? SBP6_E1(B) : (m == 2 ? SBP6_E2(B) : SBP6_E3(B));
    }
};

// support [LO, HI] of the interior edge weights (offsets of b relative to the edge's left node)
template <int O> struct EdgeRange {
    static constexpr int LO = O == 2 ? SBP2_ELO : (O == 4 ? SBP4_ELO : SBP6_ELO);
    static constexpr int HI = O == 2 ? SBP2_EHI : (O == 4 ? SBP4_EHI : SBP6_EHI);
};
// coefficient e_{m,kk} (FP32) of b_{i+kk} in E_m(i); a compile-time constant for constant m, kk
template <int O> __device__ __forceinline__ float edge_w(int m, int kk) {
    return Edge<O>::template e<float>(m, [&](int q) { return q == kk ? 1.f : 0.f; });
}

// lowest b offset used by E_m (E_m is evaluated at i only if i + elo(m) stays in range)
template <int O> __host__ __device__ constexpr int edge_lo(int m) {
    return O == 2 ? 0 : (O == 4 ? (m == 1 ? -1 : 0) : (m == 1 ? -2 : (m == 2 ? -1 : 0)));
}

// ------------------------------------------------------------------ 1-D first derivative
// D[row][col] * h  (row-major SBP operator with mirrored right closure)
template <int O> __device__ __forceinline__ double dcoef(int N, int row, int col) {
    using P = Ord<O>;
    if (row < P::NB) return (col >= 0 && col < P::NCOL) ? P::dq(row, col) : 0.0;
    if (row >= N - P::NB) {
        int r = N - 1 - row, c = N - 1 - col;
        return (c >= 0 && c < P::NCOL) ? -P::dq(r, c) : 0.0;
    }
    int k = col - row;
    if (k == 0 || k > P::Q || k < -P::Q) return 0.0;
    return k > 0 ? P::a(k - 1) : -P::a(-k - 1);
}

// the same entry in the arithmetic type T
template <int O, typename T> __device__ __forceinline__ T dcoefT(int N, int row, int col) {
    using P = Ord<O>;
    if (row < P::NB) return (col >= 0 && col < P::NCOL) ? P::template dqT<T>(row, col) : T(0);
    if (row >= N - P::NB) {
        int r = N - 1 - row, c = N - 1 - col;
        return (c >= 0 && c < P::NCOL) ? -P::template dqT<T>(r, c) : T(0);
    }
    int k = col - row;
    if (k == 0 || k > P::Q || k < -P::Q) return T(0);
    return k > 0 ? P::template aT<T>(k - 1) : -P::template aT<T>(-k - 1);
}

// norm weight H_ii / h
template <int O> __device__ __forceinline__ double hweight(int N, int i) {
    using P = Ord<O>;
    if (i < P::NB) return P::hw(i);
    if (i >= N - P::NB) return P::hw(N - 1 - i);
    return 1.0;
}

// norm weight H_ii / h in the arithmetic type T
template <int O, typename T> __device__ __forceinline__ T hweightT(int N, int i) {
    using P = Ord<O>;
    if (i < P::NB) return P::template hwT<T>(i);
    if (i >= N - P::NB) return P::template hwT<T>(N - 1 - i);
    return T(1);
}

// first and last column of row `row` of D
template <int O> __device__ __forceinline__ void drow_range(int N, int row, int& lo, int& hi) {
    using P = Ord<O>;
    if (row < P::NB) { lo = 0; hi = P::NCOL - 1; }
    else if (row >= N - P::NB) { lo = N - P::NCOL; hi = N - 1; }
    else { lo = row - P::Q; hi = row + P::Q; }
}

// sum_j D[row][j] v(j) * h, accumulated in type T
template <int O, typename T, class F> __device__ __forceinline__ T dsum(int N, int row, F v) {
    using P = Ord<O>;
    T s = T(0);
    if (row < P::NB) {
#pragma unroll
        for (int j = 0; j < P::NCOL; ++j) s += P::template dqT<T>(row, j) * v(j);
    } else if (row >= N - P::NB) {
        const int r = N - 1 - row;
#pragma unroll
        for (int j = 0; j < P::NCOL; ++j) s -= P::template dqT<T>(r, j) * v(N - 1 - j);
    } else {
#pragma unroll
        for (int k = 1; k <= P::Q; ++k) s += P::template aT<T>(k - 1) * (v(row + k) - v(row - k));
    }
    return s;
}

// ------------------------------------------------------------------ narrow second derivative
// Row i of h^2 D_xx^FC applied to the 2-component field with the 3 coefficient fields
// (b0 = c_d1d1, b1 = c_d1d2 = c_d2d1, b2 = c_d2d2):
//   r0 += D_xx(b0) u0 + D_xx(b1) u1,   r1 += D_xx(b1) u0 + D_xx(b2) u1
template <int O, typename T, class FU0, class FU1, class FB0, class FB1, class FB2>
__device__ __forceinline__ void dxx_closure(int N, int i, FU0 u0, FU1 u1, FB0 b0, FB1 b1, FB2 b2, T& r0, T& r1) {
    using P = Ord<O>;
    const bool right = i >= N - P::NCLOS;
    const int row = right ? N - 1 - i : i;
    for (int t = P::cstart(row); t < P::cstart(row + 1); ++t) {
        int j = P::cj(t), k = P::ck(t);
        if (right) { j = N - 1 - j; k = N - 1 - k; }
        const T c = P::template ccT<T>(t);
        const T bb0 = b0(k), bb1 = b1(k), bb2 = b2(k);
        const T uu0 = u0(j), uu1 = u1(j);
        r0 += c * (bb0 * uu0 + bb1 * uu1);
        r1 += c * (bb1 * uu0 + bb2 * uu1);
    }
}
template <int O, typename T, class FU0, class FU1, class FB0, class FB1, class FB2>
__device__ __forceinline__ void dxx_interior(int i, FU0 u0, FU1 u1, FB0 b0, FB1 b1, FB2 b2, T& r0, T& r1) {
    using P = Ord<O>;
    const T uc0 = u0(i), uc1 = u1(i);
#pragma unroll
    for (int m = 1; m <= P::Q; ++m) {
        auto B0p = [&](int k) { return b0(i + k); };
        auto B1p = [&](int k) { return b1(i + k); };
        auto B2p = [&](int k) { return b2(i + k); };
        auto B0m = [&](int k) { return b0(i - m + k); };
        auto B1m = [&](int k) { return b1(i - m + k); };
        auto B2m = [&](int k) { return b2(i - m + k); };
        const T e0p = Edge<O>::template e<T>(m, B0p), e1p = Edge<O>::template e<T>(m, B1p),
                e2p = Edge<O>::template e<T>(m, B2p);
        const T e0m = Edge<O>::template e<T>(m, B0m), e1m = Edge<O>::template e<T>(m, B1m),
                e2m = Edge<O>::template e<T>(m, B2m);
        const T dp0 = u0(i + m) - uc0, dp1 = u1(i + m) - uc1;
        const T dm0 = u0(i - m) - uc0, dm1 = u1(i - m) - uc1;
        r0 += e0p * dp0 + e1p * dp1 + e0m * dm0 + e1m * dm1;
        r1 += e1p * dp0 + e2p * dp1 + e1m * dm0 + e2m * dm1;
    }
}
template <int O, typename T, class FU0, class FU1, class FB0, class FB1, class FB2>
__device__ __forceinline__ void dxx_vec(int N, int i, FU0 u0, FU1 u1, FB0 b0, FB1 b1, FB2 b2, T& r0, T& r1) {
    using P = Ord<O>;
    if (i < P::NCLOS || i >= N - P::NCLOS) dxx_closure<O, T>(N, i, u0, u1, b0, b1, b2, r0, r1);
    else dxx_interior<O, T>(i, u0, u1, b0, b1, b2, r0, r1);
}

// Closure rows of h^2 D_xx^FC(b) as matrices: row r (0 .. NCLOS-1) from the low (side 0) or high
// (side 1, mirrored) end of a line is sum_j M_b[side][r][j] u(j) with M_b[side][r][j] = sum over
// the closure triples (r, j, k) of c_rjk b(k); j, k count from that end.  b is time-independent,
// so M is formed once per material (k_closure_mats); layout [side][r][j][b0 b1 b2][line] with
// the line index (the transverse node index) fastest.
template <int O> __host__ __device__ constexpr long long closure_mat_elems(int lines) {
    return 2LL * Ord<O>::NCLOS * Ord<O>::NCLOSJ * 3 * lines;
}
// node i of a line of N nodes, through the matrices M of its direction (returns false for
// interior rows, which use the edge-weight form)
template <int O, typename T, class FU0, class FU1>
__device__ __forceinline__ bool dxx_closure_mat(int N, int i, int line, int lines, const T* __restrict__ M, FU0 u0,
                                                FU1 u1, T& r0, T& r1) {
    using P = Ord<O>;
    constexpr int NC = P::NCLOS, NJ = P::NCLOSJ;
    if (i >= NC && i < N - NC) return false;
    const int side = i >= N - NC ? 1 : 0;
    const int r = side ? N - 1 - i : i;
    const T* Mr = M + (long long)(side * NC + r) * NJ * 3 * lines + line;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int jj = side ? N - 1 - j : j;
        const T uu0 = u0(jj), uu1 = u1(jj);
        const T m0 = Mr[(long long)(3 * j) * lines], m1 = Mr[(long long)(3 * j + 1) * lines],
                m2 = Mr[(long long)(3 * j + 2) * lines];
        r0 += m0 * uu0 + m1 * uu1;
        r1 += m1 * uu0 + m2 * uu1;
    }
    return true;
}

// ------------------------------------------------------------------ views
// Coefficient planes (10), in terms of c_ijkl (0-based indices):
//  0 c0000  1 c0001  2 c0101 | 3 c1010  4 c1011  5 c1111 | 6 c0010  7 c0011  8 c0110  9 c0111
// i.e. narrow x1 (c_1j1l), narrow x2 (c_2j2l), mixed c_1j2l (plane 6 + 2j + l); c_2j1l = c_1l2j.
enum { FACE_DISP = 0, FACE_ROBIN = 1, FACE_INTF = 2 };

struct FaceDev {
    int kind, m, side, nf;
    int nbr_block, nbr_face, reversed, pad;
    double nu, hm0;           // outward reference normal component, H_m[0] (includes h_m)
    double inv_h0;            // 1 / H_m[0]
    double fac[12];           // D_m[face row][i_m] / H_m[i_m] / h_m at depth d = |i_m - face| < NCOL
    float facf[12];           // the same in FP32
    const double* jhat;       // surface scale factor per face node
    const void* ju;           // robin: J^ U (3 x nf), type T
    const void* jv;           // robin with damping: J^ V (3 x nf), type T, or null
    const void* g;            // data: displacement g (2 x K x nf) or robin J^ g, type T
    void* sat;                // scratch of k_face_sat: face term (2 x nf), normal-spread amplitude (2 x nf), type T
    void* tr;                 // interface faces: this side's trace per face node (7 x nf, type T) written by
                              // k_face_trace: u_0, u_1, traction J^ tau_0, J^ tau_1, and k c_mJmL for
                              // JL = 00, 01, 11 with k = beta d / 4 / H_m[0]; null where not kept
};

struct BlockDev {
    int n1, n2, pitch, strip;  // strip = width of the boundary strips handled by k_boundary
    int damped;               // some face has Robin damping (FaceDev::jv)
    double h1, h2;
    double ih1, ih2;          // 1 / h1, 1 / h2
    float ih1f, ih2f;         // the same in FP32 (read directly as constant operands by FP32 kernels)
    void* u[2];               // state buffers, 2 planes each
    const void* c;            // 10 planes
    const void* w;            // 1/(rho J)
    const void* jf;           // J f harmonic planes (2 x K) or null
    void* r;                  // operator output (apply mode), 2 planes
    void* du;                 // FP32 leapfrog: the increment u^n - u^{n-1} (2 planes), else null
    const double* X;          // coordinates (2 planes)
    double* G;                // metric dX_I/dx_i (4 planes, [2 i + I])
    double* J;                // Jacobian
    void* rk;                 // RK4 state (10 planes): u, v, stage velocity V, sums S_u, S_v (2 planes each)
    const void* sg;           // layer dissipation coefficient s (1 plane, type T) or null
    const void* smaps;        // strip-tile band-box tensor maps (CUtensorMap[3]: u[0], u[1], c)
    const void* mx;           // closure rows of D_xx^FC along x1 as matrices, type T (k_closure_mats)
    const void* my;           // the same along x2
    FaceDev f[4];
};

struct StepArgs {
    int cur;                  // index of the current level in BlockDev::u
    int K;                    // number of time-basis functions
    int with_data;            // include boundary data / forcing / sources
    int tstep;                // graph mode: step index inside the captured sequence
    double dt2;               // dt^2 (step mode)
    double t;                 // time of the current level
    double Tk[8];             // basis values T_k(t)
    const double* tdev;       // graph mode: device array of the times of the captured steps (else null)
    double dt;                // step size
    float dt2f;               // dt^2 in FP32
    int stage;                // RK4 mode: stage s = 1..4 of the step
    double rkh;               // RK4 mode: step size h
    float rkhf;               // the same in FP32
};

// RK4 stage epilogue (mode 2) of one node.  The classical RK4 of Sec. 7.1 on y = (u, v),
// y' = (v, a(u, t)), a = (rho J)^-1 [DD(c) u + J SAT + J f], organised by stage inputs
// Y_s = (U_s, V_s): U_1 = u, V_1 = v, U_{s+1} = u + c_{s+1} h V_s, V_{s+1} = v + c_{s+1} h a_s with
// a_s = a(U_s, t + c_s h), c = (0, 1/2, 1/2, 1), and u_new = u + h sum_s b_s V_s,
// v_new = v + h sum_s b_s a_s, b = (1, 2, 2, 1)/6.  The kernel of stage s has read U_s (state
// buffer u[cur]) and formed r = DD(c) U_s + J SAT + J f at node gi; this writes U_{s+1} (or u_new)
// into u[1 - cur] and keeps V, S_u = sum b V, S_v = sum b a and, after stage 4, (u, v) in B.rk.
// B.r holds zeros except at point-source nodes off the strips (their J f, added before the stage).
template <typename T>
__device__ __forceinline__ void rk4_store(const BlockDev& B, const StepArgs& a, size_t gi, size_t plane, T w, T r0,
                                          T r1) {
    T* __restrict__ R = reinterpret_cast<T*>(B.rk);
    T* __restrict__ Un = reinterpret_cast<T*>(B.u[1 - a.cur]);
    const int s = a.stage;
    T h;
    if constexpr (sizeof(T) == 4) h = a.rkhf; else h = a.rkh;
    // point sources off the strips were added into B.r (zero elsewhere) before this kernel ran:
    // take them into the operator sum, then clear them for the next stage
    T* __restrict__ Rs = reinterpret_cast<T*>(B.r);
    const T rs0 = Rs[gi], rs1 = Rs[plane + gi];
    if (rs0 != T(0) || rs1 != T(0)) {
        r0 += rs0;
        r1 += rs1;
        Rs[gi] = T(0);
        Rs[plane + gi] = T(0);
    }
    const T a0 = w * r0, a1 = w * r1;
    const T u0 = R[gi], u1 = R[plane + gi], v0 = R[2 * plane + gi], v1 = R[3 * plane + gi];
    const T V0 = s == 1 ? v0 : R[4 * plane + gi], V1 = s == 1 ? v1 : R[5 * plane + gi];
    const T su0 = s == 1 ? T(0) : R[6 * plane + gi], su1 = s == 1 ? T(0) : R[7 * plane + gi];
    const T sv0 = s == 1 ? T(0) : R[8 * plane + gi], sv1 = s == 1 ? T(0) : R[9 * plane + gi];
    const T b = (s == 1 || s == 4) ? T(1) / T(6) : T(1) / T(3);
    if (s < 4) {
        const T ch = s == 3 ? h : T(0.5) * h;
        Un[gi] = u0 + ch * V0;
        Un[plane + gi] = u1 + ch * V1;
        R[4 * plane + gi] = v0 + ch * a0;
        R[5 * plane + gi] = v1 + ch * a1;
        R[6 * plane + gi] = su0 + b * V0;
        R[7 * plane + gi] = su1 + b * V1;
        R[8 * plane + gi] = sv0 + b * a0;
        R[9 * plane + gi] = sv1 + b * a1;
    } else {
        const T un0 = u0 + h * (su0 + b * V0), un1 = u1 + h * (su1 + b * V1);
        Un[gi] = un0;
        Un[plane + gi] = un1;
        R[gi] = un0;
        R[plane + gi] = un1;
        R[2 * plane + gi] = v0 + h * (sv0 + b * a0);
        R[3 * plane + gi] = v1 + h * (sv1 + b * a1);
    }
}

// Dissipative Robin term (remark of Sec. 5.1: T u + U u + V u' = g) at node (i1, i2): the sum over
// the Robin faces with damping that the node lies on of J^ V / H_m[0] (the J-scaled SAT of the
// term is -(J^ V / H_m[0]) u'), as the symmetric 2 x 2 (d00, d01, d11); false if there is none.
template <typename T>
__device__ __forceinline__ bool robin_damping_at(const BlockDev& B, int i1, int i2, T& d00, T& d01, T& d11) {
    bool any = false;
    d00 = d01 = d11 = T(0);
    if (!B.damped) return false;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const FaceDev& F = B.f[f];
        if (!F.jv) continue;
        const int im = F.m == 0 ? i1 : i2, Nm = F.m == 0 ? B.n1 : B.n2;
        if ((F.side ? Nm - 1 - im : im) != 0) continue;
        const int s = F.m == 0 ? i2 : i1, nf = F.nf;
        const T* jv = reinterpret_cast<const T*>(F.jv);
        const T ih = T(F.inv_h0);
        d00 += jv[s] * ih;
        d01 += jv[nf + s] * ih;
        d11 += jv[2 * nf + s] * ih;
        any = true;
    }
    return any;
}

// the stage velocity of an RK4 stage at node gi (v for the first stage, V afterwards)
template <typename T>
__device__ __forceinline__ void rk4_stage_velocity(const BlockDev& B, const StepArgs& a, size_t gi, size_t plane, T& v0, T& v1) {
    const T* R = reinterpret_cast<const T*>(B.rk);
    const size_t o = a.stage == 1 ? 2 * plane : 4 * plane;
    v0 = R[o + gi];
    v1 = R[o + plane + gi];
}

// the per-block and per-face step constants in the arithmetic type T (FP32 kernels read the FP32
// copies, which need no conversion)
template <typename T> __device__ __forceinline__ T ih1T(const BlockDev& B) {
    if constexpr (sizeof(T) == 4) return B.ih1f; else return B.ih1;
}
template <typename T> __device__ __forceinline__ T ih2T(const BlockDev& B) {
    if constexpr (sizeof(T) == 4) return B.ih2f; else return B.ih2;
}
template <typename T> __device__ __forceinline__ T facT(const FaceDev& F, int d) {
    if constexpr (sizeof(T) == 4) return F.facf[d]; else return F.fac[d];
}
template <typename T> __device__ __forceinline__ T dt2T(const StepArgs& a) {
    if constexpr (sizeof(T) == 4) return a.dt2f; else return a.dt2;
}

// leapfrog step of one node, u^{n+1} = 2 u^n - u^{n-1} + dt^2 w r (w = 1/(rho J)), written in
// increment form: d^{n+1} = d^n + dt^2 w r, u^{n+1} = u^n + d^{n+1}, d^n = u^n - u^{n-1}.  With
// B.du (the FP32 state) the increment is a field of its own, so dt^2 w r is added to a number of
// the size of u^n - u^{n-1} instead of u^n and is not lost below half an ulp of u^n (for dt small
// against h it is of that size); without it (FP64, adjoint fields) d^n is formed from the levels.
// On a face node with the dissipative Robin term, taken with the centred velocity
// (u^{n+1} - u^{n-1}) / (2 dt), the increment solves the 2 x 2 system
// (I + al D) d^{n+1} = (I - al D) d^n + dt^2 w r, al = dt w / 2 (D from robin_damping_at).
template <typename T>
__device__ __forceinline__ void leapfrog_store(const BlockDev& B, const StepArgs& a, size_t gi, size_t plane, T u0, T u1,
                                               T wv, T r0, T r1, bool damped, T dd00, T dd01, T dd11) {
    T* __restrict__ Un = reinterpret_cast<T*>(B.u[1 - a.cur]);
    T* __restrict__ DU = reinterpret_cast<T*>(B.du);
    T v0, v1;
    if (DU) {
        v0 = DU[gi];
        v1 = DU[gi + plane];
    } else {
        v0 = u0 - Un[gi];
        v1 = u1 - Un[gi + plane];
    }
    const T f = dt2T<T>(a) * wv;
    T d0 = v0 + f * r0, d1 = v1 + f * r1;
    if (damped) {
        const T al = T(0.5 * a.dt) * wv;
        const T b0 = d0 - al * (dd00 * v0 + dd01 * v1), b1 = d1 - al * (dd01 * v0 + dd11 * v1);
        const T m00 = T(1) + al * dd00, m01 = al * dd01, m11 = T(1) + al * dd11;
        const T idet = T(1) / (m00 * m11 - m01 * m01);
        d0 = (m11 * b0 - m01 * b1) * idet;
        d1 = (m00 * b1 - m01 * b0) * idet;
    }
    Un[gi] = u0 + d0;
    Un[gi + plane] = u1 + d1;
    if (DU) {
        DU[gi] = d0;
        DU[gi + plane] = d1;
    }
}


// ------------------------------------------------------------------ mbarrier / bulk-copy helpers
// One-instruction inline-PTX wrappers (the instruction text is fixed by the PTX ISA).
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
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
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// bounded wait: returns false after `polls` unsuccessful polls or after about 2 s, whichever
// comes first (a poll may suspend the thread for a while, so the poll count alone does not bound
// the time); the clock is read only once the first poll has failed
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int polls = 1 << 30) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    for (int i = 1; i < polls; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63) == 0 && globaltimer_ns() - t0 > 2000000000ull) return false;
    }
    return false;
}
// tiled bulk tensor copy global -> shared of a 3-D box at (x, y, z); completion on `bar`
__device__ __forceinline__ void tma_load_3d(void* dst, const void* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_barrier_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// kernel error word bits (reported by the host as SBP_E_TIMEOUT)
enum { ERR_MARCH_WAIT = 4, ERR_STRIP_WAIT = 8, ERR_SELFTEST_WAIT = 16 };

}  // namespace sbp
