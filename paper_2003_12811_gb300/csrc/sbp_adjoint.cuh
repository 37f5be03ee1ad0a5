// libsbp adjoint kernels: receiver recording, misfit residuals, adjoint source injection, and the
// accumulation of the misfit gradient with respect to the transformed stiffness c and the density.
//
// The scheme is u'' = W L(c) u + W data with W = 1/(rho J) and H L symmetric (Theorems 3 and 5,
// H = H_1 (x) H_2).  For the leapfrog recursion u_{n+1} = 2u_n - u_{n-1} + dt^2 W (L u_n + data_n)
// the multipliers lambda_n of the discrete Lagrangian give psi_n = H^-1 W lambda_n, and psi obeys
// the same recursion run backwards with the homogeneous operator plus the source
// H^-1 W dPhi/du_{n+1} (the paper's remark in Sec. 5.2 that the adjoint reuses the forward solver).
// The gradient is
//   dPhi/dc_p(x) = sum_n dt^2 (H psi_n)^T dL/dc_p(x) u_n,
//   dPhi/drho(x) = -sum_n H(x) J(x) psi_n(x) . (u_{n+1} - 2u_n + u_{n-1})(x).
// L is linear in c, so dL/dc_p(x) is read off the operator term by term: the narrow rows of
// D_ii^FC(b) (closure triples and interior edge weights, Sec. 4.4), the mixed terms D_i c D_k
// (Sec. 4.6), and the SAT terms of Sec. 5.1, 5.2 and 6, which involve c only at face nodes.
#pragma once
#include "sbp_kernels.cuh"

namespace sbp {

struct GradDev {
    const void* seg;          // recomputed forward levels: level l (2 planes) at seg + l * lvl_elems
    const void* pseg;         // adjoint levels of the segment: psi level l pairs with forward level l + 1
    long long lvl_elems;
    void* gc;                 // 10 accumulator planes (dPhi/dc, plane layout of BlockDev::c)
    void* grho;               // 1 accumulator plane (dPhi/drho)
    void* gsat[4];            // per face: 7 x nf SAT contributions (planes 3m, 3m+1, 3m+2, 6..9)
    void* part;               // strip nodes: per level chunk, 11 partial sums (10 c planes, rho)
};

struct RecDev {
    int block, pad;
    long long gi;             // node offset in the planes
    double hinv;              // 1 / H at the node
};

// ------------------------------------------------------------------ receivers and misfit
template <typename T>
__global__ void k_record(const BlockDev* __restrict__ blocks, const RecDev* __restrict__ rec, int nrec, int cur,
                         double* __restrict__ out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrec) return;
    const RecDev d = rec[r];
    const BlockDev& B = blocks[d.block];
    const size_t plane = (size_t)B.n2 * B.pitch;
    const T* U = reinterpret_cast<const T*>(B.u[cur]);
    out[2 * r] = (double)U[d.gi];
    out[2 * r + 1] = (double)U[d.gi + plane];
}

// res = traces - observed per step (one CTA per step) and the per-step sum of squares
__global__ void k_residual(const double* __restrict__ tr, const double* __restrict__ obs, double* __restrict__ res,
                           int per_step, double* __restrict__ partial) {
    const size_t base = (size_t)blockIdx.x * per_step;
    double acc = 0.0;
    for (int k = threadIdx.x; k < per_step; k += blockDim.x) {
        const double r = tr[base + k] - obs[base + k];
        res[base + k] = r;
        acc += r * r;
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// out = scale * sum(partial[0..n))   (one CTA of 256 threads, fixed summation order)
__global__ void k_sum_scaled(const double* __restrict__ partial, int n, double scale, double* out) {
    double acc = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) acc += partial[k];
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = scale * red[0];
}

// psi_n += H^-1 W dt res at the receivers (receiver nodes are distinct)
template <typename T>
__global__ void k_inject(const BlockDev* __restrict__ adj, const RecDev* __restrict__ rec, int nrec, int pcur,
                         const double* __restrict__ res_row, double dt) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrec) return;
    const RecDev d = rec[r];
    const BlockDev& B = adj[d.block];
    const size_t plane = (size_t)B.n2 * B.pitch;
    T* P = reinterpret_cast<T*>(B.u[pcur]);
    const double s = d.hinv * (double)reinterpret_cast<const T*>(B.w)[d.gi] * dt;
    P[d.gi] += T(s * res_row[2 * r]);
    P[d.gi + plane] += T(s * res_row[2 * r + 1]);
}

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ void face_node(const BlockDev& B, const FaceDev& F, int s, int& i1, int& i2) {
    if (F.m == 0) { i1 = F.side ? B.n1 - 1 : 0; i2 = s; }
    else { i2 = F.side ? B.n2 - 1 : 0; i1 = s; }
}

template <int O> __device__ __forceinline__ double node_h(const BlockDev& B, int i1, int i2) {
    return B.h1 * hweight<O>(B.n1, i1) * B.h2 * hweight<O>(B.n2, i2);
}

// coefficient e_{m,kk} of b_{i+kk} in the interior edge weight E_m(i) (0 outside its support)
template <int O> __device__ __forceinline__ double edge_coef(int m, int kk) {
    return Edge<O>::template e<double>(m, [&](int q) { return q == kk ? 1.0 : 0.0; });
}

template <int O> struct GradCfg {
    // nodes at least GS from every face see only interior rows of every operator (rows within
    // Q of the node are interior narrow rows, D^T is -D there, and H = h1 h2)
    static constexpr int GS = Ord<O>::NCLOS + Ord<O>::Q;
    static_assert(GS == Ord<O>::GS, "gradient tables cover the nodes within GS of an end");
    // support of the interior edge weights E_m (offsets of b relative to the edge's left node)
    static constexpr int ELO = O == 2 ? SBP2_ELO : (O == 4 ? SBP4_ELO : SBP6_ELO);
    static constexpr int EHI = O == 2 ? SBP2_EHI : (O == 4 ? SBP4_EHI : SBP6_EHI);
};

// Gradient of the narrow rows of one grid line with respect to b at line index x, contracted with
// phi (per row) and u: s_JL = sum_rows phi_J(row) d(row of h^2 D_xx(b) u_L)/d b_x, with s01
// collecting (J, L) = (0, 1) and (1, 0).  Nodes at least GS from both ends: the edge-pair form
//   -sum_m sum_k e_{m,k} (phi(j+m) - phi(j)) (u(j+m) - u(j)),  j = x - k;
// nodes near an end: the tabulated (row, u-column, coefficient) lists (mirrored at the high end).
template <int O, typename T, class FP, class FU>
__device__ __forceinline__ void narrow_grad_line(int N, int x, FP phi, FU u, T& s00, T& s01, T& s11) {
    using P = Ord<O>;
    s00 = s01 = s11 = T(0);
    if (x >= P::GS && x < N - P::GS) {
#pragma unroll
        for (int m = 1; m <= P::Q; ++m) {
#pragma unroll
            for (int k = GradCfg<O>::ELO; k <= GradCfg<O>::EHI; ++k) {
                const double e = edge_coef<O>(m, k);
                if (e == 0.0) continue;
                const T ee = T(e);
                const int j = x - k;
                const T dp0 = phi(0, j + m) - phi(0, j), dp1 = phi(1, j + m) - phi(1, j);
                const T du0 = u(0, j + m) - u(0, j), du1 = u(1, j + m) - u(1, j);
                s00 -= ee * dp0 * du0;
                s01 -= ee * (dp0 * du1 + dp1 * du0);
                s11 -= ee * dp1 * du1;
            }
        }
        return;
    }
    const bool right = x >= N - P::GS;
    const int kk = right ? N - 1 - x : x;
    for (int t = P::gn_start(kk); t < P::gn_start(kk + 1); ++t) {
        int r = P::gn_row(t), j = P::gn_j(t);
        if (right) { r = N - 1 - r; j = N - 1 - j; }
        const T c = P::template gn_c<T>(t);
        const T p0 = phi(0, r), p1 = phi(1, r), u0 = u(0, j), u1 = u(1, j);
        s00 += c * p0 * u0;
        s01 += c * (p0 * u1 + p1 * u0);
        s11 += c * p1 * u1;
    }
}

// (D^T phi)(x) * h on a line of N nodes: -D in the interior, tabulated columns near the ends
// (the high end mirrors the low end with the sign of D flipped)
template <int O, typename T, class FP>
__device__ __forceinline__ T dt_line(int N, int x, FP phi) {
    using P = Ord<O>;
    T s = T(0);
    if (x >= P::GS && x < N - P::GS) {
#pragma unroll
        for (int k = 1; k <= P::Q; ++k) s += P::template aT<T>(k - 1) * (phi(x - k) - phi(x + k));
        return s;
    }
    const bool right = x >= N - P::GS;
    const int kk = right ? N - 1 - x : x;
    for (int t = P::dt_start(kk); t < P::dt_start(kk + 1); ++t) {
        const int r = P::dt_row(t);
        s += P::template dt_c<T>(t) * phi(right ? N - 1 - r : r);
    }
    return right ? -s : s;
}

// ------------------------------------------------------------------ SAT part of the gradient
// One thread per face node: the derivatives of (H psi)^T SAT(c, u) with respect to the c planes
// at that node (the SATs involve c only at face nodes).  For face F with normal direction m,
// tangential direction t, outward sign nu, w = u - v (interface) or u (displacement), and
// H_t = h_t hw_t(s) (H = H_m H_t on the face, H_m[0] cancels against the SAT's 1/H_m[0]):
//   normal-spread amplitude a_J = half nu c_mJmL w_L           weight  H_t sum_d D_m[face][d] psi_J(d)
//   tangential transpose    b_J = nu c_mLtJ w_L                weight  half H_t (D_t psi_J)
//   penalty                 -J^Z_JL w_L (own side and, at an interface, the neighbour's SAT,
//                            whose jump is -w)                  weight  k_own H_t (psi_J - psi^v_J)
//   traction tau_J = nu (c_mJmL D_m u_L + c_mJtL D_t u_L) in the Robin SAT (weight -H_t psi_J) and
//                    the interface average (weight -H_t (psi_J + psi^v_J) / 2)
template <typename T, int O>
__global__ void k_grad_face(const BlockDev* __restrict__ adj, const GradDev* __restrict__ gd,
                            const FaceRef* __restrict__ refs, int nrefs, int total, int nl, double beta) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const FaceRef fr = refs[find_face(refs, nrefs, t)];
    const int s = t - fr.start;
    const BlockDev& B = adj[fr.block];
    const FaceDev& F = B.f[fr.face];
    const GradDev& G = gd[fr.block];
    T* out = reinterpret_cast<T*>(G.gsat[fr.face]);
    const int nf = F.nf;
    T g[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) g[k] = T(0);
    if (F.kind != FACE_DISP && F.kind != FACE_ROBIN && F.kind != FACE_INTF) {
#pragma unroll
        for (int k = 0; k < 7; ++k) out[k * nf + s] = T(0);
        return;
    }
    const int m = F.m, n1 = B.n1, n2 = B.n2, P = B.pitch;
    const int Nm = m == 0 ? n1 : n2, Nt = m == 0 ? n2 : n1;
    const size_t plane = (size_t)n2 * P;
    const T nu = T(F.nu);
    const T ihm = (m == 0 ? ih1T<T>(B) : ih2T<T>(B)), iht = (m == 0 ? ih2T<T>(B) : ih1T<T>(B));
    const T Ht = T(m == 0 ? B.h2 : B.h1) * hweightT<O, T>(Nt, s);
    // node at tangential index sp and depth d from the face
    auto node = [&](int sp, int d) -> size_t {
        int i1, i2;
        if (m == 0) { i1 = F.side ? n1 - 1 - d : d; i2 = sp; }
        else { i2 = F.side ? n2 - 1 - d : d; i1 = sp; }
        return (size_t)i2 * P + i1;
    };
    const size_t gi = node(s, 0);
    // the neighbour's node (interface)
    const T* Pv = nullptr;
    const T* Uv = nullptr;
    size_t gv = 0, planev = 0;
    long long lv = 0;
    if (F.kind == FACE_INTF) {
        const BlockDev& V = adj[F.nbr_block];
        const FaceDev& FV = V.f[F.nbr_face];
        const GradDev& GV = gd[F.nbr_block];
        const int sv = F.reversed ? nf - 1 - s : s;
        int j1, j2;
        face_node(V, FV, sv, j1, j2);
        gv = (size_t)j2 * V.pitch + j1;
        planev = (size_t)V.n2 * V.pitch;
        Pv = reinterpret_cast<const T*>(GV.pseg);
        Uv = reinterpret_cast<const T*>(GV.seg) + GV.lvl_elems;
        lv = GV.lvl_elems;
    }
    for (int l = 0; l < nl; ++l) {
    const T* __restrict__ Ps = reinterpret_cast<const T*>(G.pseg) + (size_t)l * G.lvl_elems;
    const T* __restrict__ U = reinterpret_cast<const T*>(G.seg) + (size_t)(l + 1) * G.lvl_elems;
    const T ps0 = Ps[gi], ps1 = Ps[gi + plane];
    T pv0 = T(0), pv1 = T(0), v0 = T(0), v1 = T(0);
    if (F.kind == FACE_INTF) {
        pv0 = Pv[(size_t)l * lv + gv];
        pv1 = Pv[(size_t)l * lv + gv + planev];
        v0 = Uv[(size_t)l * lv + gv];
        v1 = Uv[(size_t)l * lv + gv + planev];
    }
    if (F.kind != FACE_DISP) {
        // traction weight Theta_J (tau enters with -Theta_J) and the derivatives of u at the node
        const T th[2] = {F.kind == FACE_ROBIN ? Ht * ps0 : T(0.5) * Ht * (ps0 + pv0),
                         F.kind == FACE_ROBIN ? Ht * ps1 : T(0.5) * Ht * (ps1 + pv1)};
        T dn[2], dtg[2];
#pragma unroll
        for (int L = 0; L < 2; ++L) {
            dn[L] = dsum<O, T>(Nm, F.side ? Nm - 1 : 0, [&](int j) { return U[node(s, F.side ? Nm - 1 - j : j) + (size_t)L * plane]; }) * ihm;
            dtg[L] = dsum<O, T>(Nt, s, [&](int j) { return U[node(j, 0) + (size_t)L * plane]; }) * iht;
        }
        // nn planes: c_mJmL with (0,1) and (1,0) sharing plane 3m+1
        g[0] -= nu * th[0] * dn[0];
        g[1] -= nu * (th[0] * dn[1] + th[1] * dn[0]);
        g[2] -= nu * th[1] * dn[1];
#pragma unroll
        for (int J = 0; J < 2; ++J)
#pragma unroll
            for (int L = 0; L < 2; ++L) g[plane_nt(m, J, L) - 6 + 3] -= nu * th[J] * dtg[L];
    }
    if (F.kind != FACE_ROBIN) {
        const bool intf = F.kind == FACE_INTF;
        const T half = intf ? T(0.5) : T(1);
        const T w0 = U[gi] - v0, w1 = U[gi + plane] - v1;
        const T w[2] = {w0, w1};
        // normal-spread weight: H_t sum_d D_m[face row][i_m] psi_J(d)  (D_m mirrored with a sign flip)
        T pa0 = T(0), pa1 = T(0);
#pragma unroll
        for (int d = 0; d < Ord<O>::NCOL; ++d) {
            const T dq = Ord<O>::template dqT<T>(0, d);
            const size_t q = node(s, d);
            pa0 += dq * Ps[q];
            pa1 += dq * Ps[q + plane];
        }
        const T sg = F.side ? T(-1) : T(1);
        pa0 *= sg * Ht * ihm;
        pa1 *= sg * Ht * ihm;
        g[0] += half * nu * pa0 * w0;
        g[1] += half * nu * (pa0 * w1 + pa1 * w0);
        g[2] += half * nu * pa1 * w1;
        // tangential transpose weight: half H_t (D_t psi_J)(s)
        const T e0 = half * Ht * iht * dsum<O, T>(Nt, s, [&](int sp) { return Ps[node(sp, 0)]; });
        const T e1 = half * Ht * iht * dsum<O, T>(Nt, s, [&](int sp) { return Ps[node(sp, 0) + plane]; });
        const T eta[2] = {e0, e1};
#pragma unroll
        for (int J = 0; J < 2; ++J)
#pragma unroll
            for (int L = 0; L < 2; ++L) g[plane_nt(m, L, J) - 6 + 3] += nu * eta[J] * w[L];
        // penalty J^Z = k_own c_mJmL (+ neighbour part)
        const double dd = 2.0;
        const T kown = T(intf ? beta * dd / 4.0 * F.inv_h0 : beta * dd * F.inv_h0);
        const T k0 = kown * Ht * (ps0 - pv0), k1 = kown * Ht * (ps1 - pv1);
        g[0] -= k0 * w0;
        g[1] -= k0 * w1 + k1 * w0;
        g[2] -= k1 * w1;
    }
    }   // levels
#pragma unroll
    for (int k = 0; k < 7; ++k) out[k * nf + s] = g[k];
}

// ------------------------------------------------------------------ bulk part of the gradient
// One node x and one level n: dL/dc_p(x) contracted with phi = H psi_n and u_n, for the narrow
// rows of both directions (planes 0-2 along x1, 3-5 along x2) and the mixed terms (planes 6-9),
// added to acc.
template <typename T, int O, bool INTERIOR>
__device__ __forceinline__ void grad_level(const BlockDev& B, const T* __restrict__ Ps, const T* __restrict__ U, int i1,
                                           int i2, T* acc) {
    using PO = Ord<O>;
    const int n1 = B.n1, n2 = B.n2, P = B.pitch;
    const size_t plane = (size_t)n2 * P;
    const T ih1 = ih1T<T>(B), ih2 = ih2T<T>(B);
    auto ps = [&](int L, int j1, int j2) { return __ldg(Ps + (size_t)L * plane + (size_t)j2 * P + j1); };
    auto uu = [&](int L, int j1, int j2) { return __ldg(U + (size_t)L * plane + (size_t)j2 * P + j1); };
    if (INTERIOR) {
        // phi = h1 h2 psi in the interior: edge-pair form of the narrow rows,
        //   dPhi/db(x) = -sum_m sum_k e_{m,k} (phi(j+m) - phi(j)) (u(j+m) - u(j)),  j = x - k
        T a00 = T(0), a01 = T(0), a11 = T(0), b00 = T(0), b01 = T(0), b11 = T(0);
#pragma unroll
        for (int m = 1; m <= PO::Q; ++m) {
#pragma unroll
            for (int k = GradCfg<O>::ELO; k <= GradCfg<O>::EHI; ++k) {
                const double e = edge_coef<O>(m, k);
                if (e == 0.0) continue;
                const T ee = T(e);
                {
                    const int j = i1 - k;
                    const T dp0 = ps(0, j + m, i2) - ps(0, j, i2), dp1 = ps(1, j + m, i2) - ps(1, j, i2);
                    const T du0 = uu(0, j + m, i2) - uu(0, j, i2), du1 = uu(1, j + m, i2) - uu(1, j, i2);
                    a00 += ee * dp0 * du0;
                    a01 += ee * (dp0 * du1 + dp1 * du0);
                    a11 += ee * dp1 * du1;
                }
                {
                    const int j = i2 - k;
                    const T dp0 = ps(0, i1, j + m) - ps(0, i1, j), dp1 = ps(1, i1, j + m) - ps(1, i1, j);
                    const T du0 = uu(0, i1, j + m) - uu(0, i1, j), du1 = uu(1, i1, j + m) - uu(1, i1, j);
                    b00 += ee * dp0 * du0;
                    b01 += ee * (dp0 * du1 + dp1 * du0);
                    b11 += ee * dp1 * du1;
                }
            }
        }
        const T hh = T(B.h1 * B.h2);
        acc[0] += -hh * ih1 * ih1 * a00;
        acc[1] += -hh * ih1 * ih1 * a01;
        acc[2] += -hh * ih1 * ih1 * a11;
        acc[3] += -hh * ih2 * ih2 * b00;
        acc[4] += -hh * ih2 * ih2 * b01;
        acc[5] += -hh * ih2 * ih2 * b11;
        // mixed: D^T = -D on interior rows
        T d1p[2], d2p[2], d1u[2], d2u[2];
#pragma unroll
        for (int L = 0; L < 2; ++L) {
            T s1 = T(0), s2 = T(0), s3 = T(0), s4 = T(0);
#pragma unroll
            for (int k = 1; k <= PO::Q; ++k) {
                const T ak = T(PO::a(k - 1));
                s1 += ak * (ps(L, i1 + k, i2) - ps(L, i1 - k, i2));
                s2 += ak * (ps(L, i1, i2 + k) - ps(L, i1, i2 - k));
                s3 += ak * (uu(L, i1 + k, i2) - uu(L, i1 - k, i2));
                s4 += ak * (uu(L, i1, i2 + k) - uu(L, i1, i2 - k));
            }
            d1p[L] = -hh * s1 * ih1;
            d2p[L] = -hh * s2 * ih2;
            d1u[L] = s3 * ih1;
            d2u[L] = s4 * ih2;
        }
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) acc[6 + 2 * a + b] += d1p[a] * d2u[b] + d2p[b] * d1u[a];
    } else {
        const T hh = T(B.h1 * B.h2);
        auto phi = [&](int L, int j1, int j2) {
            return hh * hweightT<O, T>(n1, j1) * hweightT<O, T>(n2, j2) * ps(L, j1, j2);
        };
        T s00, s01, s11;
        narrow_grad_line<O, T>(n1, i1, [&](int L, int j) { return phi(L, j, i2); }, [&](int L, int j) { return uu(L, j, i2); },
                               s00, s01, s11);
        acc[0] += s00 * ih1 * ih1;
        acc[1] += s01 * ih1 * ih1;
        acc[2] += s11 * ih1 * ih1;
        narrow_grad_line<O, T>(n2, i2, [&](int L, int j) { return phi(L, i1, j); }, [&](int L, int j) { return uu(L, i1, j); },
                               s00, s01, s11);
        acc[3] += s00 * ih2 * ih2;
        acc[4] += s01 * ih2 * ih2;
        acc[5] += s11 * ih2 * ih2;
        T d1p[2], d2p[2], d1u[2], d2u[2];
#pragma unroll
        for (int L = 0; L < 2; ++L) {
            d1p[L] = dt_line<O, T>(n1, i1, [&](int j) { return phi(L, j, i2); }) * ih1;
            d2p[L] = dt_line<O, T>(n2, i2, [&](int j) { return phi(L, i1, j); }) * ih2;
            d1u[L] = dsum<O, T>(n1, i1, [&](int j) { return uu(L, j, i2); }) * ih1;
            d2u[L] = dsum<O, T>(n2, i2, [&](int j) { return uu(L, i1, j); }) * ih2;
        }
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) acc[6 + 2 * a + b] += d1p[a] * d2u[b] + d2p[b] * d1u[a];
    }
}

// One node over the nl levels of a segment: the bulk terms of every level in registers, the SAT
// terms (summed over the segment by k_grad_face) at face nodes, then gc += dt^2 acc and
// grho -= H J sum_n psi_n . (u_{n+1} - 2 u_n + u_{n-1}).
// levels [l0, l1) of one node: bulk terms into acc[0..9], the density sum into acc[10]
template <typename T, int O, bool INTERIOR>
__device__ __forceinline__ void grad_levels(const BlockDev& B, const GradDev& G, int l0, int l1, int i1, int i2, T* acc) {
    const size_t plane = (size_t)B.n2 * B.pitch, gi = (size_t)i2 * B.pitch + i1;
    const long long lvl = G.lvl_elems;
    const T* __restrict__ PS = reinterpret_cast<const T*>(G.pseg);
    const T* __restrict__ US = reinterpret_cast<const T*>(G.seg);
    T rho = T(0);
    T um0 = US[(size_t)l0 * lvl + gi], um1 = US[(size_t)l0 * lvl + gi + plane];              // u_{n-1}
    T uc0 = US[(size_t)(l0 + 1) * lvl + gi], uc1 = US[(size_t)(l0 + 1) * lvl + gi + plane];  // u_n
    for (int l = l0; l < l1; ++l) {
        const T* Ps = PS + (size_t)l * lvl;
        const T* U = US + (size_t)(l + 1) * lvl;
        grad_level<T, O, INTERIOR>(B, Ps, U, i1, i2, acc);
        const T up0 = U[lvl + gi], up1 = U[lvl + gi + plane];
        rho += Ps[gi] * (up0 - T(2) * uc0 + um0) + Ps[gi + plane] * (up1 - T(2) * uc1 + um1);
        um0 = uc0;
        um1 = uc1;
        uc0 = up0;
        uc1 = up1;
    }
    acc[10] += rho;
}

// adds the SAT sums at face nodes, then gc += dt^2 acc[0..9], grho -= H J acc[10]
template <typename T, int O, bool INTERIOR>
__device__ __forceinline__ void grad_finish(const BlockDev& B, const GradDev& G, double dt2, int i1, int i2, T* acc) {
    const int n1 = B.n1, n2 = B.n2;
    const size_t plane = (size_t)n2 * B.pitch, gi = (size_t)i2 * B.pitch + i1;
    if (!INTERIOR) {
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const FaceDev& F = B.f[f];
            const int m = F.m;
            const int im = m == 0 ? i1 : i2, Nm = m == 0 ? n1 : n2;
            const int d = F.side ? Nm - 1 - im : im;
            if (d != 0) continue;
            const int s = m == 0 ? i2 : i1;
            const T* gs = reinterpret_cast<const T*>(G.gsat[f]);
            const int nf = F.nf;
            acc[3 * m] += gs[s];
            acc[3 * m + 1] += gs[nf + s];
            acc[3 * m + 2] += gs[2 * nf + s];
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[6 + k] += gs[(3 + k) * nf + s];
        }
    }
    T* __restrict__ GC = reinterpret_cast<T*>(G.gc);
    const T d2 = T(dt2);
#pragma unroll
    for (int p = 0; p < 10; ++p) GC[(size_t)p * plane + gi] += d2 * acc[p];
    T* __restrict__ GR = reinterpret_cast<T*>(G.grho);
    GR[gi] -= T(B.h1 * B.h2) * hweightT<O, T>(n1, i1) * hweightT<O, T>(n2, i2) * T(B.J[gi]) * acc[10];
}

template <typename T, int O>
__global__ void __launch_bounds__(256) k_grad_interior(BlockDev B, GradDev G, int nl, double dt2) {
    constexpr int GS = GradCfg<O>::GS;
    const int i1 = GS + blockIdx.x * 32 + threadIdx.x;
    const int i2 = GS + blockIdx.y * 8 + threadIdx.y;
    if (i1 >= B.n1 - GS || i2 >= B.n2 - GS) return;
    T acc[11];
#pragma unroll
    for (int p = 0; p < 11; ++p) acc[p] = T(0);
    grad_levels<T, O, true>(B, G, 0, nl, i1, i2, acc);
    grad_finish<T, O, true>(B, G, dt2, i1, i2, acc);
}

// strip node t of a block (bands of width GS along every face; side bands column by column so
// that a warp shares its distance from the face)
template <int O>
__device__ __forceinline__ void grad_strip_node(const BlockDev& B, long long t, int& i1, int& i2) {
    constexpr int S = GradCfg<O>::GS;       // every admissible block has n > 2 GS in both directions
    const int n1 = B.n1, n2 = B.n2;
    const long long top = (long long)S * n1;
    if (t < top) { i2 = (int)(t / n1); i1 = (int)(t - (long long)i2 * n1); }
    else if (t < 2 * top) { const long long u = t - top; i2 = n2 - S + (int)(u / n1); i1 = (int)(u - (long long)(i2 - n2 + S) * n1); }
    else {
        const long long u = t - 2 * top;
        const int rows = n2 - 2 * S;
        const int col = (int)(u / rows), row = (int)(u - (long long)col * rows);
        i2 = S + row;
        i1 = col < S ? col : n1 - 2 * S + col;
    }
}

// strip nodes, phase 1: level chunk blockIdx.y of nchunk; partial sums to G.part
template <typename T, int O>
__global__ void __launch_bounds__(256, 2) k_grad_strip(BlockDev B, GradDev G, int nl, int nchunk, long long nstrip) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nstrip) return;
    int i1, i2;
    grad_strip_node<O>(B, t, i1, i2);
    const int c = blockIdx.y;
    const int l0 = (int)((long long)nl * c / nchunk), l1 = (int)((long long)nl * (c + 1) / nchunk);
    T acc[11];
#pragma unroll
    for (int p = 0; p < 11; ++p) acc[p] = T(0);
    grad_levels<T, O, false>(B, G, l0, l1, i1, i2, acc);
    T* part = reinterpret_cast<T*>(G.part) + (size_t)c * 11 * nstrip;
#pragma unroll
    for (int p = 0; p < 11; ++p) part[(size_t)p * nstrip + t] = acc[p];
}

// strip nodes, phase 2: the chunks in order, the SAT sums, and the accumulator update
template <typename T, int O>
__global__ void __launch_bounds__(256) k_grad_strip_sum(BlockDev B, GradDev G, int nchunk, long long nstrip, double dt2) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nstrip) return;
    int i1, i2;
    grad_strip_node<O>(B, t, i1, i2);
    T acc[11];
#pragma unroll
    for (int p = 0; p < 11; ++p) acc[p] = T(0);
    const T* part = reinterpret_cast<const T*>(G.part);
    for (int c = 0; c < nchunk; ++c)
#pragma unroll
        for (int p = 0; p < 11; ++p) acc[p] += part[((size_t)c * 11 + p) * nstrip + t];
    grad_finish<T, O, false>(B, G, dt2, i1, i2, acc);
}

// dPhi/dC (pair layout, 10 planes of the upper triangle of M[2I+J][2K+L]) and dPhi/drho as dense
// FP64 arrays: g_C[P] = sum_p g_c[p] dc_p/dC_P with c_ijkl = J F_Ii C_IjKl F_Kk.
template <typename T>
__global__ void k_grad_to_C(BlockDev B, const T* __restrict__ gc, const T* __restrict__ grho, double* __restrict__ outC,
                            double* __restrict__ outR, int voigt) {
    const long long n = (long long)B.n1 * B.n2;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int i2 = (int)(t / B.n1), i1 = (int)(t - (long long)i2 * B.n1);
    const size_t P = B.pitch, plane = (size_t)B.n2 * P, gi = (size_t)i2 * P + i1;
    const double g00 = B.G[gi], g01 = B.G[plane + gi], g10 = B.G[2 * plane + gi], g11 = B.G[3 * plane + gi];
    const double J = B.J[gi];
    double F[2][2];
    F[0][0] = g11 / J;
    F[0][1] = -g01 / J;
    F[1][0] = -g10 / J;
    F[1][1] = g00 / J;
    double g[10];
    for (int p = 0; p < 10; ++p) g[p] = (double)gc[(size_t)p * plane + gi];
    const int ijkl[10][4] = {{0, 0, 0, 0}, {0, 0, 0, 1}, {0, 1, 0, 1}, {1, 0, 1, 0}, {1, 0, 1, 1},
                             {1, 1, 1, 1}, {0, 0, 1, 0}, {0, 0, 1, 1}, {0, 1, 1, 0}, {0, 1, 1, 1}};
    // Voigt output (minor symmetry): the Voigt entry of pair entry idx (the Voigt index of a pair
    // p = 2I+J is 0 for (0,0), 1 for (1,1), 2 for (0,1)/(1,0); upper triangle in the order
    // 11 12 13 22 23 33); a Voigt entry moves every pair entry that maps to it, so its derivative
    // is the sum of theirs
    const int to_voigt[10] = {0, 2, 2, 1, 5, 5, 4, 5, 4, 3};
    double gv[6] = {0, 0, 0, 0, 0, 0};
    int idx = 0;
    for (int p = 0; p < 4; ++p)
        for (int q = p; q < 4; ++q) {
            // unit pair entry (p, q) and its mirror
            double s = 0.0;
            for (int pl = 0; pl < 10; ++pl) {
                const int i = ijkl[pl][0], j = ijkl[pl][1], k = ijkl[pl][2], l = ijkl[pl][3];
                double c = 0.0;
                for (int I = 0; I < 2; ++I)
                    for (int K = 0; K < 2; ++K) {
                        const int a = 2 * I + j, b = 2 * K + l;
                        if ((a == p && b == q) || (a == q && b == p)) c += F[I][i] * F[K][k];
                    }
                s += g[pl] * J * c;
            }
            if (voigt) gv[to_voigt[idx]] += s;
            else outC[(size_t)idx * n + t] = s;
            ++idx;
        }
    if (voigt)
        for (int v = 0; v < 6; ++v) outC[(size_t)v * n + t] = gv[v];
    outR[t] = (double)grho[gi];
}

}  // namespace sbp
