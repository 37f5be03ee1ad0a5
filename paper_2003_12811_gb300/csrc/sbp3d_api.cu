// libsbp 3-D operator: host implementation of include/sbp3.h (handle, validation, device memory,
// material setup, leapfrog step loop, apply).  The kernels are in sbp3d.cuh.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/sbp3.h"
#include "sbp3d.cuh"

using namespace sbp3;

namespace {

thread_local std::string g3_create_error;

constexpr int NCM = 27, NCD = 18;

int min_nodes(int order) { return order == 2 ? 5 : (order == 4 ? 18 : 27); }

struct Prof {
    std::vector<cudaEvent_t> ev[SBP3_PROF_FAMILIES];   // start/stop pairs
    double ms[SBP3_PROF_FAMILIES] = {0, 0, 0};
};

}  // namespace

struct sbp3_handle {
    int order = 0, precision = 0;
    int n[3] = {0, 0, 0};
    long long pitch = 0, fs = 0;
    size_t es = 8;
    double beta = 1.0;
    Grid3 g{};
    Box3 box{};                              // nodes with interior rows in every direction (k3_div_int)
    long long shell = 0;                     // nodes outside the box (k3_div_shell)
    Shell3 sh{};
    Faces3 fc{};
    int div_variant = 0;                     // launch shape of k3_div_int (kDivShapes)
    double* X = nullptr;                     // pitched FP64 coordinates (3 fields)
    void* cm = nullptr;                      // 27 fields
    void* cd = nullptr;                      // 18 fields
    void* w = nullptr;                       // 1 field
    void* u[2] = {nullptr, nullptr};         // leapfrog levels (3 fields each), u[cur] = u^n
    void* du = nullptr;                      // increment u^n - u^{n-1} (3 fields)
    void* q = nullptr;                       // mixed fluxes (9 fields)
    void* xm = nullptr;                      // x1 closure matrices of D_xx^FC (k3_xclos)
    void* ain = nullptr;                     // sbp3_apply input / output (3 fields each), on first use
    void* aout = nullptr;
    int cur = 0;
    std::vector<char> planes_set;
    long long nplanes_set = 0;
    bool state = false;
    int* d_err = nullptr;
    int device = 0;
    bool prof_on = false;
    Prof prof;
    long long launches[SBP3_PROF_FAMILIES] = {0, 0, 0};
    std::string err;
};

namespace {

int fail(sbp3_handle* h, int code, const std::string& m) {
    if (h) h->err = m;
    else g3_create_error = m;
    return code;
}

int cuda_fail(sbp3_handle* h, cudaError_t e, const char* where) {
    return fail(h, SBP_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK3(h, call)                                                                         \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) return e_ == cudaErrorMemoryAllocation ? fail(h, SBP_E_OOM, #call) : cuda_fail(h, e_, #call); \
    } while (0)

long long pitch_of(int n1, size_t es) {
    const long long q = 128 / (long long)es;
    return (n1 + q - 1) / q * q;
}

struct DeviceGuard {
    int prev = 0;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (ok) cudaSetDevice(prev);
    }
};

void prof_begin(sbp3_handle* h, int fam, cudaStream_t st, cudaEvent_t* stop) {
    *stop = nullptr;
    ++h->launches[fam];
    if (!h->prof_on) return;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, st);
    h->prof.ev[fam].push_back(a);
    h->prof.ev[fam].push_back(b);
    *stop = b;
}

void prof_end(cudaEvent_t stop, cudaStream_t st) {
    if (stop) cudaEventRecord(stop, st);
}

template <typename T, int O, int MODE>
int launch_operator(sbp3_handle* h, const T* u, T* du, T* un, double dt, cudaStream_t st) {
    const Grid3& g = h->g;
    constexpr int NVF = sizeof(T) == 4 ? 2 : 1;
    const dim3 blk(BX, BY), grd((g.n[0] + BX * NVF - 1) / (BX * NVF), (g.n[1] + BY - 1) / BY, g.n[2]);
    const T* cm = static_cast<const T*>(h->cm);
    const T* cd = static_cast<const T*>(h->cd);
    const T* w = static_cast<const T*>(h->w);
    T* q = static_cast<T*>(h->q);
    const T dt2 = T(dt * dt);
    cudaEvent_t stop;
    prof_begin(h, 0, st, &stop);
    k3_flux<T, O, NVF><<<grd, blk, 0, st>>>(g, u, cm, q);
    prof_end(stop, st);
    {
        constexpr int NV = sizeof(T) == 4 ? 2 : 1;
        const Box3& bx = h->box;
        const int ngx = (bx.x1hi - bx.x1lo) / NV;
        if (ngx > 0) {             // the box is empty only for order 2 on the smallest grids
            auto run = [&](auto vc) {
                constexpr int V = decltype(vc)::value;
                constexpr int BY = kDivShapes[V].by, MINB = kDivShapes[V].minb;
                const dim3 ib(32, BY), ig((ngx + 31) / 32, (bx.y1 - bx.y0 + BY - 1) / BY, bx.z1 - bx.z0);
                k3_div_int<T, O, MODE, NV, BY, MINB><<<ig, ib, 0, st>>>(g, bx, h->fc, u, q, cm, cd, w, du, un, dt2);
            };
            prof_begin(h, 1, st, &stop);
            // every shape is built for order 6; orders 2 and 4 keep the first
            const int v = O == 6 ? h->div_variant : 0;
            if (v == 1) run(std::integral_constant<int, O == 6 ? 1 : 0>());
            else if (v == 2) run(std::integral_constant<int, O == 6 ? 2 : 0>());
            else if (v == 3) run(std::integral_constant<int, O == 6 ? 3 : 0>());
            else run(std::integral_constant<int, 0>());
            prof_end(stop, st);
        }
        const long long cnt = h->shell;
        prof_begin(h, 2, st, &stop);
        const XClos xc{h->xm, (long long)h->n[1] * h->n[2]};
        k3_div_shell<T, O, MODE><<<(unsigned)((cnt + 127) / 128), 128, 0, st>>>(g, bx, h->sh, xc, h->fc, cnt, u, q,
                                                                             cm, cd, w, du, un, dt2);
        prof_end(stop, st);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "3-D operator launch");
    return SBP_OK;
}

template <typename T, int O>
int step_impl(sbp3_handle* h, int nsteps, double dt, cudaStream_t st) {
    for (int s = 0; s < nsteps; ++s) {
        T* uc = static_cast<T*>(h->u[h->cur]);
        T* un = static_cast<T*>(h->u[1 - h->cur]);
        int rc = launch_operator<T, O, 0>(h, uc, static_cast<T*>(h->du), un, dt, st);
        if (rc != SBP_OK) return rc;
        h->cur = 1 - h->cur;
    }
    return SBP_OK;
}

template <typename T, int O>
int apply_impl(sbp3_handle* h, cudaStream_t st) {
    return launch_operator<T, O, 1>(h, static_cast<const T*>(h->ain), nullptr, static_cast<T*>(h->aout), 0.0, st);
}

template <typename T, int O>
int material_impl(sbp3_handle* h, int k0, int nk, const double* rho_d, const double* c_d) {
    const dim3 blk(128), grd((h->n[0] + 127) / 128, h->n[1], nk);
    k3_material<T, O><<<grd, blk>>>(h->g, h->X, k0, nk, rho_d, c_d, static_cast<T*>(h->cm), static_cast<T*>(h->cd),
                                     static_cast<T*>(h->w), h->d_err);
    const dim3 xg((h->n[1] + 127) / 128, nk, 2 * Ord<O>::NCLOS);
    k3_xclos<T, O><<<xg, 128>>>(h->g, k0, nk, static_cast<const T*>(h->cd), static_cast<T*>(h->xm));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "k3_material");
    return SBP_OK;
}

template <typename F> int dispatch(sbp3_handle* h, F f) {
    // f(T tag, order constant)
    if (h->precision == SBP_FP64) {
        switch (h->order) {
            case 2: return f(double(), std::integral_constant<int, 2>());
            case 4: return f(double(), std::integral_constant<int, 4>());
            default: return f(double(), std::integral_constant<int, 6>());
        }
    }
    switch (h->order) {
        case 2: return f(float(), std::integral_constant<int, 2>());
        case 4: return f(float(), std::integral_constant<int, 4>());
        default: return f(float(), std::integral_constant<int, 6>());
    }
}

void free_all(sbp3_handle* h) {
    void* bufs[] = {h->X, h->cm, h->cd, h->w, h->u[0], h->u[1], h->du, h->q, h->xm, h->ain, h->aout, h->d_err};
    for (void* b : bufs)
        if (b) cudaFree(b);
    for (auto& v : h->prof.ev)
        for (cudaEvent_t e : v)
            if (e) cudaEventDestroy(e);
}

size_t xclos_bytes(int order, size_t es, int n2, int n3) {
    const int nclos = order == 2 ? SBP2_NCLOS : (order == 4 ? SBP4_NCLOS : SBP6_NCLOS);
    const int nj = order == 2 ? SBP2_NCLOSJ : (order == 4 ? SBP4_NCLOSJ : SBP6_NCLOSJ);
    return (size_t)2 * nj * 6 * nclos * (size_t)n2 * n3 * es;
}

long long field_bytes(int precision, const int n[3]) {
    const size_t es = precision == SBP_FP32 ? 4 : 8;
    return pitch_of(n[0], es) * n[1] * n[2] * (long long)es;
}

bool check_range(const sbp3_handle* h) {
    return h && h->nplanes_set == h->n[2];
}

}  // namespace

extern "C" {

const char* sbp3_last_error(const sbp3_handle* h) { return h ? h->err.c_str() : g3_create_error.c_str(); }

int sbp3_footprint(int order, int precision, int n1, int n2, int n3, long long* bytes_out) {
    if (!bytes_out || n1 <= 0 || n2 <= 0 || n3 <= 0 || (precision != SBP_FP64 && precision != SBP_FP32) ||
        (order != 2 && order != 4 && order != 6))
        return fail(nullptr, SBP_E_INVALID_ARG, "sbp3_footprint: bad arguments");
    const int n[3] = {n1, n2, n3};
    const long long f = field_bytes(precision, n);
    const long long x = pitch_of(n1, precision == SBP_FP32 ? 4 : 8) * n2 * n3 * 8LL;
    *bytes_out = f * (NCM + NCD + 1 + 6 + 3 + 9) + 3 * x +
                 (long long)xclos_bytes(order, precision == SBP_FP32 ? 4 : 8, n2, n3);
    return SBP_OK;
}

int sbp3_create(int order, int precision, int n1, int n2, int n3, const double* X, const int* face_kinds,
                double beta, sbp3_handle** out) {
    g3_create_error.clear();
    if (!out) return fail(nullptr, SBP_E_INVALID_ARG, "sbp3_create: out is NULL");
    *out = nullptr;
    if (order != 2 && order != 4 && order != 6) return fail(nullptr, SBP_E_INVALID_ARG, "order must be 2, 4 or 6");
    if (precision != SBP_FP64 && precision != SBP_FP32) return fail(nullptr, SBP_E_INVALID_ARG, "bad precision");
    const int mn = min_nodes(order);
    if (n1 < mn || n2 < mn || n3 < mn)
        return fail(nullptr, SBP_E_INVALID_ARG, "need n1, n2, n3 >= " + std::to_string(mn) + " for order " +
                                                    std::to_string(order));
    if (n3 > 65535 || n2 > 65535) return fail(nullptr, SBP_E_INVALID_ARG, "n2, n3 must be <= 65535");
    // neighbour offsets are 32-bit: up to 16 planes away from a node must stay below 2^31 elements
    if (pitch_of(n1, precision == SBP_FP32 ? 4 : 8) * (long long)n2 * 16 >= (1LL << 31))
        return fail(nullptr, SBP_E_INVALID_ARG, "an x3-plane must hold fewer than 2^27 elements");
    if (!X || !face_kinds) return fail(nullptr, SBP_E_INVALID_ARG, "X and face_kinds are required");
    for (int f = 0; f < 6; ++f)
        if (face_kinds[f] != SBP3_BC_DISPLACEMENT && face_kinds[f] != SBP3_BC_TRACTION)
            return fail(nullptr, SBP_E_INVALID_ARG, "face kind must be SBP3_BC_DISPLACEMENT or SBP3_BC_TRACTION");
    if (!(beta > 0.0) || !std::isfinite(beta)) return fail(nullptr, SBP_E_INVALID_ARG, "beta must be positive");
    const long long N = (long long)n1 * n2 * n3;
    for (long long i = 0; i < 3 * N; ++i)
        if (!std::isfinite(X[i])) return fail(nullptr, SBP_E_INVALID_ARG, "X has a non-finite value");

    sbp3_handle* h = new sbp3_handle();
    h->order = order;
    h->precision = precision;
    h->n[0] = n1;
    h->n[1] = n2;
    h->n[2] = n3;
    h->es = precision == SBP_FP32 ? 4 : 8;
    h->pitch = pitch_of(n1, h->es);
    h->fs = h->pitch * n2 * n3;
    h->beta = beta;
    for (int f = 0; f < 6; ++f) h->fc.kind[f] = face_kinds[f];
    h->fc.beta = beta;
    h->planes_set.assign(n3, 0);
    cudaGetDevice(&h->device);
    Grid3& g = h->g;
    for (int i = 0; i < 3; ++i) {
        g.n[i] = h->n[i];
        g.ih[i] = double(h->n[i] - 1);
    }
    g.s[0] = 1;
    g.s[1] = h->pitch;
    g.s[2] = h->pitch * n2;
    g.fs = h->fs;
    {
        const int nclos = order == 2 ? SBP2_NCLOS : (order == 4 ? SBP4_NCLOS : SBP6_NCLOS);
        const int q = order / 2, nv = precision == SBP_FP32 ? 2 : 1;
        const int qa = (q + nv - 1) / nv * nv;            // the x1 window of k3_div_int reaches qa nodes out
        const int ncol = order == 2 ? SBP2_NCOL : (order == 4 ? SBP4_NCOL : SBP6_NCOL);
        // the shell holds every node with a closure row, a normal SAT term (depth < NCOL) or an x1
        // window of k3_div_int that would leave the row
        const int ey = nclos > ncol ? nclos : ncol;
        const int e = ey > qa ? ey : qa;
        Box3& bx = h->box;
        bx.x1lo = (e + nv - 1) / nv * nv;
        bx.x1hi = n1 - e > bx.x1lo ? bx.x1lo + (n1 - e - bx.x1lo) / nv * nv : bx.x1lo;
        bx.y0 = 0;
        bx.y1 = n2;
        bx.z0 = 0;
        bx.z1 = n3;
        Shell3& sh = h->sh;
        sh.cZ = (long long)(bx.z0 + (n3 - bx.z1)) * n2 * n1;
        sh.cY = (long long)(bx.z1 - bx.z0) * (bx.y0 + (n2 - bx.y1)) * n1;
        sh.cX = (long long)(bx.z1 - bx.z0) * (bx.y1 - bx.y0) * (bx.x1lo + (n1 - bx.x1hi));
        h->shell = sh.cX + sh.cZ + sh.cY;
    }
    auto alloc = [&](void** p, size_t bytes) -> bool {
        if (cudaMalloc(p, bytes) != cudaSuccess) return false;
        return cudaMemset(*p, 0, bytes) == cudaSuccess;
    };
    const size_t fb = (size_t)h->fs * h->es;
    // the FP64 coordinates share the element pitch of the T fields (a multiple of 16 elements)
    const long long xp = h->pitch;
    const size_t xfs = (size_t)h->fs;
    bool ok = alloc((void**)&h->X, 3 * xfs * 8) && alloc(&h->cm, NCM * fb) && alloc(&h->cd, NCD * fb) &&
              alloc(&h->w, fb) && alloc(&h->u[0], 3 * fb) && alloc(&h->u[1], 3 * fb) && alloc(&h->du, 3 * fb) &&
              alloc(&h->q, 9 * fb) && alloc(&h->xm, xclos_bytes(order, h->es, n2, n3)) &&
              alloc((void**)&h->d_err, sizeof(int));
    if (!ok) {
        cudaGetLastError();
        free_all(h);
        delete h;
        return fail(nullptr, SBP_E_OOM, "sbp3_create: device allocation failed");
    }
    for (int I = 0; I < 3; ++I) {
        cudaError_t e = cudaMemcpy2D(h->X + I * xfs, xp * 8, X + I * N, (size_t)n1 * 8, (size_t)n1 * 8,
                                     (size_t)n2 * n3, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            free_all(h);
            delete h;
            return fail(nullptr, SBP_E_CUDA, std::string("sbp3_create: ") + cudaGetErrorString(e));
        }
    }
    *out = h;
    return SBP_OK;
}

int sbp3_destroy(sbp3_handle* h) {
    if (!h) return SBP_E_INVALID_ARG;
    DeviceGuard dg(h->device);
    cudaDeviceSynchronize();
    free_all(h);
    delete h;
    return SBP_OK;
}

int sbp3_set_material(sbp3_handle* h, int i3_begin, int i3_count, const double* rho, const double* C45) {
    if (!h) return fail(nullptr, SBP_E_INVALID_ARG, "null handle");
    if (!rho || !C45 || i3_begin < 0 || i3_count <= 0 || i3_begin + i3_count > h->n[2])
        return fail(h, SBP_E_INVALID_ARG, "sbp3_set_material: bad plane range or null array");
    const long long np = (long long)h->n[0] * h->n[1] * i3_count;
    for (long long i = 0; i < np; ++i)
        if (!(rho[i] > 0.0) || !std::isfinite(rho[i])) return fail(h, SBP_E_INVALID_ARG, "rho must be positive");
    for (long long i = 0; i < 45 * np; ++i)
        if (!std::isfinite(C45[i])) return fail(h, SBP_E_INVALID_ARG, "C45 has a non-finite value");
    DeviceGuard dg(h->device);
    double* buf = nullptr;
    CK3(h, cudaMalloc(&buf, 46 * np * sizeof(double)));
    cudaError_t e = cudaMemcpy(buf, rho, np * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(buf + np, C45, 45 * np * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(h->d_err, 0, sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(buf);
        return cuda_fail(h, e, "sbp3_set_material upload");
    }
    int rc = dispatch(h, [&](auto tag, auto oc) {
        using T = decltype(tag);
        constexpr int O = decltype(oc)::value;
        return material_impl<T, O>(h, i3_begin, i3_count, buf, buf + np);
    });
    int herr = 0;
    e = cudaMemcpy(&herr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (rc != SBP_OK) return rc;
    if (e != cudaSuccess) return cuda_fail(h, e, "sbp3_set_material");
    if (herr) return fail(h, SBP_E_JACOBIAN_NONPOSITIVE, "J <= 0 at a node of the given planes");
    for (int k = i3_begin; k < i3_begin + i3_count; ++k) {
        if (!h->planes_set[k]) ++h->nplanes_set;
        h->planes_set[k] = 1;
    }
    return SBP_OK;
}

int sbp3_set_state(sbp3_handle* h, const double* u_prev, const double* u_cur) {
    if (!h) return fail(nullptr, SBP_E_INVALID_ARG, "null handle");
    if (!u_prev || !u_cur) return fail(h, SBP_E_INVALID_ARG, "sbp3_set_state: null array");
    const long long N = (long long)h->n[0] * h->n[1] * h->n[2];
    DeviceGuard dg(h->device);
    double* buf = nullptr;
    CK3(h, cudaMalloc(&buf, 6 * N * sizeof(double)));
    cudaError_t e = cudaMemcpy(buf, u_prev, 3 * N * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(buf + 3 * N, u_cur, 3 * N * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(buf);
        return cuda_fail(h, e, "sbp3_set_state upload");
    }
    const dim3 blk(128), grd((h->n[0] + 127) / 128, h->n[1], h->n[2]);
    if (h->precision == SBP_FP32)
        k3_load_state<float><<<grd, blk>>>(h->g, buf, buf + 3 * N, (float*)h->u[1 - h->cur], (float*)h->u[h->cur],
                                            (float*)h->du);
    else
        k3_load_state<double><<<grd, blk>>>(h->g, buf, buf + 3 * N, (double*)h->u[1 - h->cur],
                                             (double*)h->u[h->cur], (double*)h->du);
    e = cudaDeviceSynchronize();
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(h, e, "k3_load_state");
    h->state = true;
    return SBP_OK;
}

int sbp3_get_state(sbp3_handle* h, double* u_prev, double* u_cur) {
    if (!h) return fail(nullptr, SBP_E_INVALID_ARG, "null handle");
    if (!u_prev || !u_cur) return fail(h, SBP_E_INVALID_ARG, "sbp3_get_state: null array");
    if (!h->state) return fail(h, SBP_E_STATE, "no state set");
    const long long N = (long long)h->n[0] * h->n[1] * h->n[2];
    DeviceGuard dg(h->device);
    double* buf = nullptr;
    CK3(h, cudaMalloc(&buf, 6 * N * sizeof(double)));
    const dim3 blk(128), grd((h->n[0] + 127) / 128, h->n[1], h->n[2]);
    if (h->precision == SBP_FP32) {
        k3_store_field<float><<<grd, blk>>>(h->g, (const float*)h->u[1 - h->cur], buf);
        k3_store_field<float><<<grd, blk>>>(h->g, (const float*)h->u[h->cur], buf + 3 * N);
    } else {
        k3_store_field<double><<<grd, blk>>>(h->g, (const double*)h->u[1 - h->cur], buf);
        k3_store_field<double><<<grd, blk>>>(h->g, (const double*)h->u[h->cur], buf + 3 * N);
    }
    cudaError_t e = cudaMemcpy(u_prev, buf, 3 * N * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(u_cur, buf + 3 * N, 3 * N * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(h, e, "sbp3_get_state");
    return SBP_OK;
}

int sbp3_apply(sbp3_handle* h, const double* u, double* accel) {
    if (!h) return fail(nullptr, SBP_E_INVALID_ARG, "null handle");
    if (!u || !accel) return fail(h, SBP_E_INVALID_ARG, "sbp3_apply: null array");
    if (!check_range(h)) return fail(h, SBP_E_STATE, "material not set for every x3-plane");
    const long long N = (long long)h->n[0] * h->n[1] * h->n[2];
    DeviceGuard dg(h->device);
    const size_t fb = (size_t)h->fs * h->es;
    if (!h->ain) CK3(h, cudaMalloc(&h->ain, 3 * fb));
    if (!h->aout) CK3(h, cudaMalloc(&h->aout, 3 * fb));
    double* buf = nullptr;
    CK3(h, cudaMalloc(&buf, 3 * N * sizeof(double)));
    cudaError_t e = cudaMemcpy(buf, u, 3 * N * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(buf);
        return cuda_fail(h, e, "sbp3_apply upload");
    }
    const dim3 blk(128), grd((h->n[0] + 127) / 128, h->n[1], h->n[2]);
    if (h->precision == SBP_FP32) k3_load_field<float><<<grd, blk>>>(h->g, buf, (float*)h->ain);
    else k3_load_field<double><<<grd, blk>>>(h->g, buf, (double*)h->ain);
    int rc = dispatch(h, [&](auto tag, auto oc) {
        using T = decltype(tag);
        constexpr int O = decltype(oc)::value;
        return apply_impl<T, O>(h, 0);
    });
    if (rc != SBP_OK) {
        cudaFree(buf);
        return rc;
    }
    if (h->precision == SBP_FP32) k3_store_field<float><<<grd, blk>>>(h->g, (const float*)h->aout, buf);
    else k3_store_field<double><<<grd, blk>>>(h->g, (const double*)h->aout, buf);
    e = cudaMemcpy(accel, buf, 3 * N * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(h, e, "sbp3_apply");
    return SBP_OK;
}

int sbp3_step(sbp3_handle* h, int nsteps, double dt, void* stream) {
    if (!h) return fail(nullptr, SBP_E_INVALID_ARG, "null handle");
    if (nsteps < 0 || !(dt > 0.0) || !std::isfinite(dt)) return fail(h, SBP_E_INVALID_ARG, "bad nsteps or dt");
    if (!check_range(h)) return fail(h, SBP_E_STATE, "material not set for every x3-plane");
    if (!h->state) return fail(h, SBP_E_STATE, "no state set");
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return dispatch(h, [&](auto tag, auto oc) {
        using T = decltype(tag);
        constexpr int O = decltype(oc)::value;
        return step_impl<T, O>(h, nsteps, dt, st);
    });
}

int sbp3_set_tuning(sbp3_handle* h, int variant) {
    if (!h) return fail(nullptr, SBP_E_INVALID_ARG, "null handle");
    if (variant < 0 || variant >= SBP3_TUNING_VARIANTS) return fail(h, SBP_E_INVALID_ARG, "bad tuning variant");
    h->div_variant = h->order == 6 ? variant : 0;
    return SBP_OK;
}

int sbp3_autotune(sbp3_handle* h, int* variant_out, double* ms_out) {
    if (!h) return fail(nullptr, SBP_E_INVALID_ARG, "null handle");
    if (!check_range(h)) return fail(h, SBP_E_STATE, "material not set for every x3-plane");
    DeviceGuard dg(h->device);
    const size_t fb = (size_t)h->fs * h->es;
    if (!h->ain) CK3(h, cudaMalloc(&h->ain, 3 * fb));
    if (!h->aout) CK3(h, cudaMalloc(&h->aout, 3 * fb));
    // operator applications on the current level (or on zeros before any state): the state is untouched
    if (h->state) CK3(h, cudaMemcpy(h->ain, h->u[h->cur], 3 * fb, cudaMemcpyDeviceToDevice));
    else CK3(h, cudaMemset(h->ain, 0, 3 * fb));
    const int nv = h->order == 6 ? SBP3_TUNING_VARIANTS : 1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const bool prof = h->prof_on;
    h->prof_on = false;
    int best = 0;
    double best_ms = 1e300;
    for (int v = 0; v < nv; ++v) {
        h->div_variant = v;
        int rc = SBP_OK;
        for (int rep = 0; rep < 2 && rc == SBP_OK; ++rep)
            rc = dispatch(h, [&](auto tag, auto oc) {
                using T = decltype(tag);
                constexpr int O = decltype(oc)::value;
                return apply_impl<T, O>(h, 0);
            });
        cudaEventRecord(e0, 0);
        for (int rep = 0; rep < 5 && rc == SBP_OK; ++rep)
            rc = dispatch(h, [&](auto tag, auto oc) {
                using T = decltype(tag);
                constexpr int O = decltype(oc)::value;
                return apply_impl<T, O>(h, 0);
            });
        cudaEventRecord(e1, 0);
        cudaError_t e = cudaEventSynchronize(e1);
        if (rc != SBP_OK || e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            h->prof_on = prof;
            h->div_variant = 0;
            return rc != SBP_OK ? rc : cuda_fail(h, e, "sbp3_autotune");
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (ms_out) ms_out[v] = t / 5.0;
        if (t < best_ms) {
            best_ms = t;
            best = v;
        }
    }
    for (int v = nv; v < SBP3_TUNING_VARIANTS; ++v)
        if (ms_out) ms_out[v] = -1.0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->prof_on = prof;
    h->div_variant = best;
    if (variant_out) *variant_out = best;
    return SBP_OK;
}

int sbp3_profile(sbp3_handle* h, int enable) {
    if (!h) return fail(nullptr, SBP_E_INVALID_ARG, "null handle");
    h->prof_on = enable != 0;
    return SBP_OK;
}

int sbp3_profile_read(sbp3_handle* h, double* ms, long long* launches) {
    if (!h || !ms || !launches) return fail(h, SBP_E_INVALID_ARG, "sbp3_profile_read: null argument");
    DeviceGuard dg(h->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(h, e, "sbp3_profile_read");
    for (int f = 0; f < SBP3_PROF_FAMILIES; ++f) {
        auto& v = h->prof.ev[f];
        for (size_t i = 0; i + 1 < v.size(); i += 2) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, v[i], v[i + 1]) == cudaSuccess) h->prof.ms[f] += t;
            cudaEventDestroy(v[i]);
            cudaEventDestroy(v[i + 1]);
        }
        v.clear();
        ms[f] = h->prof.ms[f];
        launches[f] = h->launches[f];
    }
    return SBP_OK;
}

int sbp3_get_info(const sbp3_handle* h, long long* nodes_out, int* precision_out, int* order_out) {
    if (!h) return SBP_E_INVALID_ARG;
    if (nodes_out) *nodes_out = (long long)h->n[0] * h->n[1] * h->n[2];
    if (precision_out) *precision_out = h->precision;
    if (order_out) *order_out = h->order;
    return SBP_OK;
}

}  // extern "C"
