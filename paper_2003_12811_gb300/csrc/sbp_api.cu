// libsbp host implementation: handle, validation, device memory, setup and the leapfrog step
// loop.  The declarations and their documentation are in include/sbp.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "../../include/sbp.h"
#include "sbp_interior_march.cuh"
#include "sbp_kernels.cuh"
#include "sbp_adjoint.cuh"
#include "sbp_batch.cuh"
#include "sbp_wide.cuh"

namespace sbphost {
#define SBP_TABLE static const
#include "sbp_tables.inc"
#undef SBP_TABLE
}  // namespace sbphost

using namespace sbp;

namespace {

thread_local std::string g_create_error;

struct HostFace {
    int kind = -1, nbr_block = -1, nbr_face = -1, reversed = 0;
    int nf = 0;
    double* jhat = nullptr;
    void* ju = nullptr;
    void* g = nullptr;
    void* sat = nullptr;      // wide stencil: SAT terms of the face nodes (k_face_sat); else unused (sbp_apply_noalloc
                              // points its views at its own scratch)
    void* tr = nullptr;       // interface faces: trace of this side (k_face_trace), 7 x nf
    void* jv = nullptr;       // Robin faces with damping: J^ V (3 x nf, type T)
};

struct HostBlock {
    int n1 = 0, n2 = 0, pitch = 0;
    double h1 = 0, h2 = 0;
    void* u[2] = {nullptr, nullptr};
    void* du = nullptr;       // FP32: the leapfrog increment u^n - u^{n-1} (2 planes)
    void* c = nullptr;
    void* w = nullptr;
    void* jf = nullptr;
    void* r = nullptr;
    double* X = nullptr;
    double* G = nullptr;
    double* J = nullptr;
    bool material = false;
    HostFace f[4];
    MarchMaps mmaps;          // FP32 column-marching interior kernel tensor maps
    void* psi[2] = {nullptr, nullptr};   // adjoint fields (sbp_misfit_gradient), allocated on first use
    MarchMaps pmaps;          // marching-kernel maps over the adjoint fields
    CUtensorMap* d_smaps = nullptr;   // strip-tile band-box maps on the device: [0..2] state u0, u1, c; [3..5] adjoint
    void* rk = nullptr;       // RK4 state (u, v, V, S_u, S_v; sbp_set_state_rk4), allocated on first use
    void* gw = nullptr;       // wide stencil: the fluxes G_1j, G_2j (4 planes, type T)
    void* sg = nullptr;       // layer dissipation coefficient s (1 plane, type T)
    int2* d_lnodes = nullptr; // nodes the layer dissipation reaches, (i1, i2)
    int nln = 0;
    void* lscr = nullptr;     // leapfrog: the dissipation of the listed nodes between the pre and post kernels
    void* mx = nullptr;       // closure matrices of D_xx^FC along x1 / x2 (k_closure_mats, type T)
    void* my = nullptr;
};

int order_nb(int o) { return o == 2 ? SBP2_NB : (o == 4 ? SBP4_NB : SBP6_NB); }
int order_ncol(int o) { return o == 2 ? SBP2_NCOL : (o == 4 ? SBP4_NCOL : SBP6_NCOL); }
int order_nclos(int o) { return o == 2 ? SBP2_NCLOS : (o == 4 ? SBP4_NCLOS : SBP6_NCLOS); }
int order_nclosj(int o) { return o == 2 ? SBP2_NCLOSJ : (o == 4 ? SBP4_NCLOSJ : SBP6_NCLOSJ); }
// elements of the closure matrices of one direction with `lines` lines (layout of dxx_closure_mat)
size_t closure_elems(int o, int lines) { return 2 * (size_t)order_nclos(o) * order_nclosj(o) * 3 * lines; }
int order_q(int o) { return o / 2; }
int order_min_n(int o) { return o == 2 ? 5 : (o == 4 ? 18 : 27); }
double order_hw(int o, int i) {
    return o == 2 ? sbphost::sbp2_HW[i] : (o == 4 ? sbphost::sbp4_HW[i] : sbphost::sbp6_HW[i]);
}
double order_dq0(int o, int c) {
    return o == 2 ? sbphost::sbp2_DQ[0][c] : (o == 4 ? sbphost::sbp4_DQ[0][c] : sbphost::sbp6_DQ[0][c]);
}
double host_hweight(int o, int N, int i) {
    const int nb = order_nb(o);
    if (i < nb) return order_hw(o, i);
    if (i >= N - nb) return order_hw(o, N - 1 - i);
    return 1.0;
}

}  // namespace

struct sbp_handle {
    int order = 0, precision = 0, nblocks = 0;
    int stencil = SBP_STENCIL_NARROW;
    bool layers = false;          // some block has layer dissipation (sbp_set_layer_dissipation)
    bool damping = false;         // some face has Robin damping or some block layers
    double beta = 1.0;
    size_t esize = 8;
    std::vector<HostBlock> blocks;
    BlockDev* d_blocks = nullptr;
    FaceRef* d_refs = nullptr;
    int nrefs = 0, nface_nodes = 0;
    int ntrefs = 0;               // interface faces (their traces: k_face_trace)
    int cur = 0;
    double t = 0.0;
    int nbasis = 0;
    int basis_kind[8] = {0};
    double basis_omega[8] = {0};
    std::vector<SrcNode> src_nodes;
    std::vector<SrcParam> src_params;
    SrcNode* d_src_nodes = nullptr;     // every source node (sbp_apply_noalloc)
    SrcNode* d_src_int = nullptr;       // source nodes off the boundary strips (k_sources)
    int n_src_int = 0;
    SrcNode* d_src_strip = nullptr;     // source nodes on the strips, grouped by strip tile (k_strip_tile)
    SrcParam* d_src_params = nullptr;
    bool src_dirty = false;
    double* d_scalar = nullptr;
    int* d_flag = nullptr;
    int* d_err = nullptr;       // kernel error flags (bounded waits that ran out)
    int num_sms = 0;
    int device = 0;             // CUDA device current at sbp_grid_create (holds every buffer)
    std::string err;
    std::vector<void*> allocs;
    // kernel timing (benchmarks): the families of sbp_profile in include/sbp.h
    bool prof = false;
    double prof_ms[SBP_PROF_FAMILIES] = {0};
    long long launches[SBP_PROF_FAMILIES] = {0};
    std::vector<cudaEvent_t> ev_pool;
    struct Pending { int fam; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    // CUDA-graph step loop (sbp_step_graph): graph of `graph_steps` steps of size `graph_dt`
    cudaGraphExec_t graph_exec = nullptr;
    int graph_steps = 0;
    double graph_dt = 0.0;
    double* d_time = nullptr;     // device copies of the step times of a graph launch
    int d_time_cap = 0;
    // marching-kernel rows per CTA chosen by sbp_autotune (0 = default heuristic)
    int rows_per_cta = 0;
    // optionally (sbp_autotune, sbp_set_tuning) the boundary strips run on a second stream
    // concurrently with the interior kernel (they write disjoint nodes); both are forked from and
    // joined back into the launch stream every step, the interior on a high-priority stream so
    // that its CTAs are placed first
    bool overlap = false;
    cudaStream_t hi = nullptr;
    cudaEvent_t ev_join_hi = nullptr;
    // strip tiles of every block, costliest first (one k_strip_tile launch per step)
    int4* d_tiles = nullptr;            // (block, tile, first, end source node of the tile) in launch order
    int ntiles = 0;
    std::vector<int4> tiles_host;
    std::vector<std::vector<int>> tile_pos;   // [block][tile of the block] -> position in the launch order
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // adjoint: block views whose state buffers are the adjoint fields; receivers
    BlockDev* d_blocks_adj = nullptr;
    std::vector<RecDev> recs;
    RecDev* d_recs = nullptr;

    cudaEvent_t get_event() {
        if (!ev_pool.empty()) {
            cudaEvent_t e = ev_pool.back();
            ev_pool.pop_back();
            return e;
        }
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }

    int fail(int code, const std::string& msg) {
        err = msg;
        return code;
    }
    // one grow-only device staging buffer for host uploads and downloads: setup and transfer calls
    // use it instead of allocating and freeing temporaries (a free synchronises the whole device,
    // which would stall work other streams run meanwhile, e.g. a batch of served shots)
    void* stage = nullptr;
    size_t stage_bytes = 0;
    void* staging(size_t bytes) {
        if (bytes <= stage_bytes) return stage;
        if (stage) dfree(stage);
        stage = dalloc(bytes + bytes / 4);
        stage_bytes = stage ? bytes + bytes / 4 : 0;
        return stage;
    }
    void* dalloc(size_t bytes) {
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
        cudaMemset(p, 0, bytes);
        allocs.push_back(p);
        return p;
    }
    void dfree(void* p) {
        if (!p) return;
        allocs.erase(std::remove(allocs.begin(), allocs.end(), p), allocs.end());
        cudaFree(p);
    }
};

namespace {

// records CUDA events around one kernel family when profiling is on; counts launches always
struct ProfScope {
    sbp_handle* h;
    int fam;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(sbp_handle* h_, int fam_, cudaStream_t st_, int nlaunch) : h(h_), fam(fam_), st(st_) {
        h->launches[fam] += nlaunch;
        if (h->prof) {
            a = h->get_event();
            b = h->get_event();
            cudaEventRecord(a, st);
        }
    }
    ~ProfScope() {
        if (h->prof) {
            cudaEventRecord(b, st);
            h->pending.push_back({fam, a, b});
        }
    }
};

int check_cuda(sbp_handle* h, const char* where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return h->fail(SBP_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
    return SBP_OK;
}

BlockDev make_view(const sbp_handle* h, const HostBlock& hb) {
    BlockDev b{};
    b.n1 = hb.n1;
    b.n2 = hb.n2;
    b.pitch = hb.pitch;
    b.strip = std::max(order_nclos(h->order), order_ncol(h->order));
    b.h1 = hb.h1;
    b.h2 = hb.h2;
    b.ih1 = 1.0 / hb.h1;
    b.ih2 = 1.0 / hb.h2;
    b.ih1f = (float)b.ih1;
    b.ih2f = (float)b.ih2;
    b.u[0] = hb.u[0];
    b.u[1] = hb.u[1];
    b.du = hb.du;
    b.c = hb.c;
    b.w = hb.w;
    b.jf = hb.jf;
    b.r = hb.r;
    b.X = hb.X;
    b.G = hb.G;
    b.J = hb.J;
    for (int f = 0; f < 4; ++f) {
        const HostFace& F = hb.f[f];
        FaceDev& D = b.f[f];
        D.kind = F.kind;
        D.m = f / 2;
        D.side = f % 2;
        D.nf = F.nf;
        D.nbr_block = F.nbr_block;
        D.nbr_face = F.nbr_face;
        D.reversed = F.reversed;
        D.nu = (f % 2 == 0) ? -1.0 : 1.0;
        const int Nm = (f / 2 == 0) ? hb.n1 : hb.n2;
        const double hm = (f / 2 == 0) ? hb.h1 : hb.h2;
        D.hm0 = hm * host_hweight(h->order, Nm, 0);
        D.inv_h0 = 1.0 / D.hm0;
        // D_m[face row][i_m] / (h_m^2 hw(i_m)) at depth d: the boundary row of D (mirrored with the
        // opposite sign at the high end) over the norm weight
        for (int d = 0; d < 12; ++d) {
            const double dq0 = d < order_ncol(h->order) ? order_dq0(h->order, d) : 0.0;
            D.fac[d] = ((f % 2) ? -dq0 : dq0) / (hm * hm * host_hweight(h->order, Nm, (f % 2) ? Nm - 1 - d : d));
            D.facf[d] = (float)D.fac[d];
        }
        D.jhat = F.jhat;
        D.ju = F.ju;
        D.g = F.g;
        D.sat = F.sat;
        D.tr = F.tr;
        D.jv = F.jv;
        if (F.jv) b.damped = 1;
    }
    b.smaps = hb.d_smaps;
    b.rk = hb.rk;
    b.sg = hb.sg;
    b.mx = hb.mx;
    b.my = hb.my;
    return b;
}

// the same view with the adjoint fields as its state buffers
BlockDev make_view_adj(const sbp_handle* h, const HostBlock& hb) {
    BlockDev b = make_view(h, hb);
    b.u[0] = hb.psi[0];
    b.u[1] = hb.psi[1];
    b.du = nullptr;             // the adjoint fields step from their two levels
    b.smaps = hb.d_smaps ? hb.d_smaps + 3 : nullptr;
    return b;
}

int sync_views(sbp_handle* h) {
    std::vector<BlockDev> v;
    for (auto& hb : h->blocks) v.push_back(make_view(h, hb));
    if (cudaMemcpy(h->d_blocks, v.data(), sizeof(BlockDev) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return h->fail(SBP_E_CUDA, "upload of block views failed");
    if (h->d_blocks_adj) {
        v.clear();
        for (auto& hb : h->blocks) v.push_back(make_view_adj(h, hb));
        if (cudaMemcpy(h->d_blocks_adj, v.data(), sizeof(BlockDev) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return h->fail(SBP_E_CUDA, "upload of adjoint block views failed");
    }
    return SBP_OK;
}

inline unsigned grid_for(long long n, int bs = 256) { return (unsigned)((n + bs - 1) / bs); }

// the FP32 leapfrog increment of a block re-formed from its two levels (after the levels were
// written by something other than a leapfrog step)
void refresh_increment(sbp_handle* h, const HostBlock& hb, cudaStream_t st) {
    if (!hb.du) return;
    const long long n = 2LL * hb.n2 * hb.pitch;
    k_diff_levels<<<grid_for(n), 256, 0, st>>>((float*)hb.du, (const float*)hb.u[h->cur], (const float*)hb.u[1 - h->cur], n);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 3-D map over `planes` consecutive float planes of n2 x pitch, box [planes][rows][width]
bool make_map(CUtensorMap* m, void* base, int pitch, int n2, int planes, int rows, int width, int esize = 4) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)pitch, (cuuint64_t)n2, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)pitch * esize, (cuuint64_t)pitch * n2 * esize};
    cuuint32_t box[3] = {(cuuint32_t)width, (cuuint32_t)rows, (cuuint32_t)planes};
    cuuint32_t estr[3] = {1, 1, 1};
    return fn(m, esize == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides,
              box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// strip-tile band box of the block's order (tiles along x1)
template <int O> void strip_box(int& bw, int& bh) {
    bw = StripTile<O>::BWB;
    bh = StripTile<O>::BHB;
}

// the strip-tile band-box maps of two displacement buffers and the coefficients, written to dst[0..2]
bool make_strip_maps(const sbp_handle* h, const HostBlock& hb, void* u0, void* u1, CUtensorMap* dst) {
    int bw, bh;
    if (h->order == 2) strip_box<2>(bw, bh);
    else if (h->order == 4) strip_box<4>(bw, bh);
    else strip_box<6>(bw, bh);
    const int es = (int)h->esize;
    return make_map(&dst[0], u0, hb.pitch, hb.n2, 2, bh, bw, es) &&
           make_map(&dst[1], u1, hb.pitch, hb.n2, 2, bh, bw, es) &&
           make_map(&dst[2], hb.c, hb.pitch, hb.n2, 10, bh, bw, es);
}

// interface traces of the level being read (k_face_trace), TRACE_MAX faces per launch, on stream tst
template <typename T, int O>
void launch_traces(sbp_handle* h, const StepArgs& a, cudaStream_t tst, bool adj) {
    TraceArgs ta{};
    auto flush = [&]() {
        if (ta.nfaces == 0) return;
        ProfScope ps(h, 2, tst, 1);
        k_face_trace<T, O><<<grid_for(ta.total, 128), 128, 0, tst>>>(ta);
        ta = TraceArgs{};
    };
    for (size_t b = 0; b < h->blocks.size(); ++b) {
        const HostBlock& hb = h->blocks[b];
        for (int f = 0; f < 4; ++f) {
            const HostFace& HF = hb.f[f];
            if (HF.kind != FACE_INTF) continue;
            TraceFace& F = ta.f[ta.nfaces++];
            F.u = adj ? hb.psi[a.cur] : hb.u[a.cur];
            F.c = hb.c;
            F.tr = HF.tr;
            F.plane = (long long)hb.n2 * hb.pitch;
            F.nf = HF.nf;
            F.start = ta.total;
            F.m = f / 2;
            F.side = f % 2;
            F.pitch = hb.pitch;
            F.nm = F.m == 0 ? hb.n1 : hb.n2;
            F.nu = (f % 2 == 0) ? -1.0 : 1.0;
            const double hm = F.m == 0 ? hb.h1 : hb.h2, ht = F.m == 0 ? hb.h2 : hb.h1;
            F.ihm = 1.0 / hm;
            F.iht = 1.0 / ht;
            F.k = h->beta * 2.0 / 4.0 * (1.0 / (hm * host_hweight(h->order, F.nm, 0)));
            ta.total += HF.nf;
            if (ta.nfaces == TRACE_MAX) flush();
        }
    }
    flush();
}

// the wide-stencil operator (sbp_wide.cuh): traces, the SAT terms of every face node, the flux and
// divergence passes of every block, then the point sources (every source node: the wide path has
// no strip kernel); RK4 stages take the sources into the operator sum first
template <typename T, int O>
int launch_wide(sbp_handle* h, const StepArgs& a, int mode, cudaStream_t st) {
    if (!h->src_nodes.empty() && mode == 2) {
        ProfScope ps(h, 3, st, 1);
        const int ns = (int)h->src_nodes.size();
        k_sources<T, 2><<<grid_for(ns), 256, 0, st>>>(h->d_blocks, h->d_src_nodes, ns, h->d_src_params, a);
    }
    if (h->ntrefs > 0) launch_traces<T, O>(h, a, st, false);
    if (h->nface_nodes > 0) {
        ProfScope ps(h, 1, st, 1);
        k_face_sat<T, O><<<grid_for(h->nface_nodes), 256, 0, st>>>(h->d_blocks, h->d_refs, h->nrefs, h->nface_nodes, a, h->beta);
    }
    for (auto& hb : h->blocks) {
        const BlockDev b = make_view(h, hb);
        const long long n = (long long)hb.n1 * hb.n2;
        ProfScope ps(h, 0, st, 2);
        k_wide_flux<T, O><<<grid_for(n), 256, 0, st>>>(b, a, (T*)hb.gw);
        if (mode == 0) k_wide_div<T, O, 0><<<grid_for(n), 256, 0, st>>>(b, a, (const T*)hb.gw);
        else if (mode == 2) k_wide_div<T, O, 2><<<grid_for(n), 256, 0, st>>>(b, a, (const T*)hb.gw);
        else k_wide_div<T, O, 1><<<grid_for(n), 256, 0, st>>>(b, a, (const T*)hb.gw);
    }
    if (!h->src_nodes.empty() && mode != 2) {
        ProfScope ps(h, 3, st, 1);
        const int ns = (int)h->src_nodes.size();
        if (mode == 0) k_sources<T, 0><<<grid_for(ns), 256, 0, st>>>(h->d_blocks, h->d_src_nodes, ns, h->d_src_params, a);
        else k_sources<T, 1><<<grid_for(ns), 256, 0, st>>>(h->d_blocks, h->d_src_nodes, ns, h->d_src_params, a);
    }
    return check_cuda(h, "wide operator launch");
}

// one operator application (mode 1) or leapfrog step (mode 0) on the state fields, or, with adj,
// on the adjoint fields (the same kernels; the sources are skipped)
template <typename T, int O>
int launch_operator(sbp_handle* h, const StepArgs& a, int mode, cudaStream_t st, bool adj) {
    const BlockDev* tab = adj ? h->d_blocks_adj : h->d_blocks;
    constexpr size_t smem = interior_smem_elems<T, O>() * sizeof(T);
    // interior kernels on st; strip kernels on the auxiliary stream when overlapping (profiling
    // runs serialise so that every family's events time that family alone)
    if (mode == 2 && !adj && h->n_src_int > 0) {   // RK4 stage: interior sources first (into r)
        ProfScope ps(h, 3, st, 1);
        k_sources<T, 2><<<grid_for(h->n_src_int), 256, 0, st>>>(h->d_blocks, h->d_src_int, h->n_src_int, h->d_src_params, a);
    }
    const bool ovl = h->overlap && h->aux && !h->prof;
    // the interface traces run on the auxiliary stream beside the interior kernel (in its tail
    // or its free slots); the strips that read them follow on that stream or wait for it
    const bool tr_async = h->aux && !h->prof && h->ntrefs > 0;
    cudaStream_t sst = ovl ? h->aux : st;
    cudaStream_t ist = ovl ? h->hi : st;
    cudaStream_t tst = (ovl || tr_async) ? h->aux : st;
    if (ovl || tr_async) {
        cudaEventRecord(h->ev_fork, st);
        cudaStreamWaitEvent(h->aux, h->ev_fork, 0);
        if (ovl) cudaStreamWaitEvent(h->hi, h->ev_fork, 0);
    }
    if constexpr (std::is_same<T, float>::value) {
        // column-marching kernel: the interior tiles of up to MARCH_MAX_BLOCKS blocks per launch,
        // rows per tile chosen for one wave of ~4 CTAs per SM per block
        MarchMulti mmul{};
        int tiles = 0;
        auto flush = [&]() {
            if (mmul.nb == 0) return;
            mmul.start[mmul.nb] = tiles;
            ProfScope ps(h, 0, ist, 1);
            constexpr size_t msm = MarchCfg<O>::BYTES;
            if (mode == 0 && !adj) k_interior_march_multi<O, 3><<<tiles, MTHREADS, msm, ist>>>(mmul, a, h->d_err);
            else if (mode == 0) k_interior_march_multi<O, 0><<<tiles, MTHREADS, msm, ist>>>(mmul, a, h->d_err);
            else if (mode == 2) k_interior_march_multi<O, 2><<<tiles, MTHREADS, msm, ist>>>(mmul, a, h->d_err);
            else k_interior_march_multi<O, 1><<<tiles, MTHREADS, msm, ist>>>(mmul, a, h->d_err);
            mmul = MarchMulti{};
            tiles = 0;
        };
        for (auto& hb : h->blocks) {
            const int S2 = std::max(order_nclos(h->order), order_ncol(h->order));
            const int ncx = march_ncx(hb.n1, S2);
            const int n2i = hb.n2 - 2 * S2;
            int ncy = std::max(1, (4 * h->num_sms + ncx / 2) / ncx);
            int rows = (n2i + ncy - 1) / ncy;
            if (rows < 16) rows = std::min(16, n2i);
            if (h->rows_per_cta > 0) rows = std::min(h->rows_per_cta, n2i);
            ncy = (n2i + rows - 1) / rows;
            const int k = mmul.nb++;
            mmul.maps[k] = adj ? hb.pmaps : hb.mmaps;
            mmul.b[k] = adj ? make_view_adj(h, hb) : make_view(h, hb);
            mmul.start[k] = tiles;
            mmul.rows[k] = rows;
            tiles += ncx * ncy;
            if (mmul.nb == MARCH_MAX_BLOCKS) flush();
        }
        flush();
    } else for (auto& hb : h->blocks) {
        BlockDev b = adj ? make_view_adj(h, hb) : make_view(h, hb);
        const int S = b.strip;
        const int ni1 = hb.n1 - 2 * S, ni2 = hb.n2 - 2 * S;
        dim3 grid((ni1 + ITX - 1) / ITX, (ni2 + ITY - 1) / ITY);
        {
            ProfScope ps(h, 0, ist, 1);
            {
                if (mode == 0) k_interior<T, O, 0><<<grid, dim3(32, 8), smem, ist>>>(b, a);
                else if (mode == 2) k_interior<T, O, 2><<<grid, dim3(32, 8), smem, ist>>>(b, a);
                else k_interior<T, O, 1><<<grid, dim3(32, 8), smem, ist>>>(b, a);
            }
        }
    }
    if (h->ntrefs > 0) launch_traces<T, O>(h, a, tst, adj);
    if (tr_async && !ovl) {    // the strips wait for the traces formed beside the interior
        cudaEventRecord(h->ev_join, h->aux);
        cudaStreamWaitEvent(st, h->ev_join, 0);
    }
    {
        ProfScope ps(h, 1, sst, 1);
        using ST = StripTile<O>;
        constexpr size_t ssm = ST::template bytes<T>();
        const SrcNode* ss = adj ? nullptr : h->d_src_strip;
        if (mode == 0)
            k_strip_tile<T, O, 0><<<h->ntiles, ST::THREADS, ssm, sst>>>(tab, h->d_tiles, a, h->beta, h->d_err, ss, h->d_src_params);
        else if (mode == 2)
            k_strip_tile<T, O, 2><<<h->ntiles, ST::THREADS, ssm, sst>>>(tab, h->d_tiles, a, h->beta, h->d_err, ss, h->d_src_params);
        else
            k_strip_tile<T, O, 1><<<h->ntiles, ST::THREADS, ssm, sst>>>(tab, h->d_tiles, a, h->beta, h->d_err, ss, h->d_src_params);
    }
    if (ovl) {
        cudaEventRecord(h->ev_join, h->aux);
        cudaEventRecord(h->ev_join_hi, h->hi);
        cudaStreamWaitEvent(st, h->ev_join, 0);
        cudaStreamWaitEvent(st, h->ev_join_hi, 0);
    }
    if (!adj && h->n_src_int > 0 && mode != 2) {   // source nodes off the strips (the strip kernel adds the others)
        ProfScope ps(h, 3, st, 1);
        const int ns = h->n_src_int;
        if (mode == 0) k_sources<T, 0><<<grid_for(ns), 256, 0, st>>>(h->d_blocks, h->d_src_int, ns, h->d_src_params, a);
        else k_sources<T, 1><<<grid_for(ns), 256, 0, st>>>(h->d_blocks, h->d_src_int, ns, h->d_src_params, a);
    }
    return check_cuda(h, "operator launch");
}

template <typename T>
int dispatch_operator(sbp_handle* h, const StepArgs& a, int mode, cudaStream_t st, bool adj) {
    if (h->stencil == SBP_STENCIL_WIDE) {
        switch (h->order) {
            case 2: return launch_wide<T, 2>(h, a, mode, st);
            case 4: return launch_wide<T, 4>(h, a, mode, st);
            default: return launch_wide<T, 6>(h, a, mode, st);
        }
    }
    switch (h->order) {
        case 2: return launch_operator<T, 2>(h, a, mode, st, adj);
        case 4: return launch_operator<T, 4>(h, a, mode, st, adj);
        default: return launch_operator<T, 6>(h, a, mode, st, adj);
    }
}

// layer dissipation around the step kernels (leapfrog: the backward-velocity term is formed before
// the step overwrites u^{n-1} and added after it; RK4: added into the stage's operator sum before)
template <typename T, int O>
void layer_launch(sbp_handle* h, const StepArgs& a, int mode, cudaStream_t st, bool post) {
    if (mode == 0 && !(a.dt > 0)) return;   // tuning steps advance nothing (dt = 0)
    for (auto& hb : h->blocks) {
        if (hb.nln == 0) continue;
        const BlockDev b = make_view(h, hb);
        const unsigned g = grid_for(hb.nln);
        if (mode == 2) {
            if (!post) k_layer_rk<T, O><<<g, 256, 0, st>>>(b, hb.d_lnodes, hb.nln, a.stage);
        } else if (!post) {
            k_layer_pre<T, O><<<g, 256, 0, st>>>(b, hb.d_lnodes, hb.nln, a.cur, 1.0 / a.dt, (T*)hb.lscr);
        } else {
            k_layer_post<T><<<g, 256, 0, st>>>(b, hb.d_lnodes, hb.nln, a.cur, a.dt, (const T*)hb.lscr);
        }
    }
}

void run_layers(sbp_handle* h, const StepArgs& a, int mode, cudaStream_t st, bool post) {
    if (h->precision == SBP_FP64) {
        if (h->order == 2) layer_launch<double, 2>(h, a, mode, st, post);
        else if (h->order == 4) layer_launch<double, 4>(h, a, mode, st, post);
        else layer_launch<double, 6>(h, a, mode, st, post);
    } else {
        if (h->order == 2) layer_launch<float, 2>(h, a, mode, st, post);
        else if (h->order == 4) layer_launch<float, 4>(h, a, mode, st, post);
        else layer_launch<float, 6>(h, a, mode, st, post);
    }
}

int run_operator(sbp_handle* h, const StepArgs& a, int mode, cudaStream_t st, bool adj = false) {
    const bool layers = !adj && h->layers && (mode == 0 || mode == 2);
    if (layers) run_layers(h, a, mode, st, false);
    const int rc = h->precision == SBP_FP64 ? dispatch_operator<double>(h, a, mode, st, adj)
                                            : dispatch_operator<float>(h, a, mode, st, adj);
    if (rc == SBP_OK && layers && mode == 0) run_layers(h, a, mode, st, true);
    return rc;
}

template <typename T, int O> void set_smem_attr() {
    constexpr size_t smem = interior_smem_elems<T, O>() * sizeof(T);
    constexpr size_t ssm = StripTile<O>::template bytes<T>();
    cudaFuncSetAttribute(k_strip_tile<T, O, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm);
    cudaFuncSetAttribute(k_strip_tile<T, O, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm);
    cudaFuncSetAttribute(k_strip_tile<T, O, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm);
    cudaFuncSetAttribute(k_interior<T, O, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_interior<T, O, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_interior<T, O, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (std::is_same<T, float>::value) {
        cudaFuncSetAttribute(k_interior_march<O, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MarchCfg<O>::BYTES);
        cudaFuncSetAttribute(k_interior_march<O, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MarchCfg<O>::BYTES);
        cudaFuncSetAttribute(k_interior_march<O, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MarchCfg<O>::BYTES);
        cudaFuncSetAttribute(k_interior_march_multi<O, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MarchCfg<O>::BYTES);
        cudaFuncSetAttribute(k_interior_march_multi<O, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MarchCfg<O>::BYTES);
        cudaFuncSetAttribute(k_interior_march_multi<O, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MarchCfg<O>::BYTES);
        cudaFuncSetAttribute(k_interior_march_multi<O, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MarchCfg<O>::BYTES);
    }
}

// kernel error word: ERR_* bits (sbp_device.cuh) set by kernels whose bounded wait ran out
int check_kernel_errors(sbp_handle* h) {
    int e = 0;
    if (cudaMemcpy(&e, h->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return h->fail(SBP_E_CUDA, std::string("device error: ") + cudaGetErrorString(cudaGetLastError()));
    if (e) {
        cudaMemset(h->d_err, 0, sizeof(int));
        return h->fail(SBP_E_TIMEOUT, "a bounded wait in a kernel ran out; results of the last steps are invalid");
    }
    return SBP_OK;
}

void fill_basis(const sbp_handle* h, double t, StepArgs& a) {
    a.K = h->nbasis;
    for (int k = 0; k < h->nbasis; ++k) a.Tk[k] = h->basis_kind[k] == 0 ? sin(h->basis_omega[k] * t) : cos(h->basis_omega[k] * t);
}

// strip tile of node (i1, i2) of a block in the numbering of k_strip_tile (bands of width S along
// x2 = 0 and x2 = 1, then the side bands between them), or -1 for a node off the strips
int strip_tile_of(const sbp_handle* h, const HostBlock& hb, int i1, int i2) {
    const int S = std::max(order_nclos(h->order), order_ncol(h->order));
    const int nbx = (hb.n1 + 31) / 32, nby = (hb.n2 - 2 * S + 31) / 32;
    if (i2 < S) return i1 / 32;
    if (i2 >= hb.n2 - S) return nbx + i1 / 32;
    if (i1 < S) return 2 * nbx + (i2 - S) / 32;
    if (i1 >= hb.n1 - S) return 2 * nbx + nby + (i2 - S) / 32;
    return -1;
}

int upload_sources(sbp_handle* h) {
    if (!h->src_dirty) return SBP_OK;
    h->dfree(h->d_src_nodes);
    h->dfree(h->d_src_params);
    h->dfree(h->d_src_int);
    h->dfree(h->d_src_strip);
    h->d_src_int = h->d_src_strip = nullptr;
    h->n_src_int = 0;
    h->d_src_nodes = (SrcNode*)h->dalloc(sizeof(SrcNode) * h->src_nodes.size());
    h->d_src_params = (SrcParam*)h->dalloc(sizeof(SrcParam) * h->src_params.size());
    if (!h->d_src_nodes || !h->d_src_params) return h->fail(SBP_E_OOM, "source tables");
    if (cudaMemcpy(h->d_src_nodes, h->src_nodes.data(), sizeof(SrcNode) * h->src_nodes.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->d_src_params, h->src_params.data(), sizeof(SrcParam) * h->src_params.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return h->fail(SBP_E_CUDA, "source table upload failed");
    // split: nodes on the boundary strips go with their strip tile, the rest to k_sources
    std::vector<std::pair<int, SrcNode>> strip;
    std::vector<SrcNode> inner;
    for (const SrcNode& nd : h->src_nodes) {
        const HostBlock& hb = h->blocks[nd.block];
        const int i2 = (int)(nd.gi / hb.pitch), i1 = (int)(nd.gi - (long long)i2 * hb.pitch);
        const int t = strip_tile_of(h, hb, i1, i2);
        if (t < 0) inner.push_back(nd);
        else strip.push_back({h->tile_pos[nd.block][t], nd});
    }
    std::stable_sort(strip.begin(), strip.end(),
                     [](const std::pair<int, SrcNode>& x, const std::pair<int, SrcNode>& y) { return x.first < y.first; });
    for (int4& tl : h->tiles_host) tl.z = tl.w = 0;
    std::vector<SrcNode> sv;
    for (size_t k = 0; k < strip.size(); ++k) {
        int4& tl = h->tiles_host[strip[k].first];
        if (tl.z == tl.w) tl.z = tl.w = (int)k;
        tl.w = (int)k + 1;
        sv.push_back(strip[k].second);
    }
    if (!sv.empty()) {
        h->d_src_strip = (SrcNode*)h->dalloc(sizeof(SrcNode) * sv.size());
        if (!h->d_src_strip) return h->fail(SBP_E_OOM, "source tables");
        if (cudaMemcpy(h->d_src_strip, sv.data(), sizeof(SrcNode) * sv.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return h->fail(SBP_E_CUDA, "source table upload failed");
    }
    if (!inner.empty()) {
        h->d_src_int = (SrcNode*)h->dalloc(sizeof(SrcNode) * inner.size());
        if (!h->d_src_int) return h->fail(SBP_E_OOM, "source tables");
        if (cudaMemcpy(h->d_src_int, inner.data(), sizeof(SrcNode) * inner.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return h->fail(SBP_E_CUDA, "source table upload failed");
        h->n_src_int = (int)inner.size();
    }
    if (cudaMemcpy(h->d_tiles, h->tiles_host.data(), sizeof(int4) * h->tiles_host.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return h->fail(SBP_E_CUDA, "tile table upload failed");
    if (h->graph_exec) {   // captured launches hold the old tables and launch counts
        cudaGraphExecDestroy(h->graph_exec);
        h->graph_exec = nullptr;
    }
    h->src_dirty = false;
    return check_cuda(h, "source upload");
}

bool all_materials(const sbp_handle* h) {
    for (auto& b : h->blocks)
        if (!b.material) return false;
    return true;
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// Fixed scratch for sbp_apply_noalloc.  Callers that cannot allocate device memory (for example
// code running inside a memory pool it may not grow, or a real-time loop where cudaMalloc's
// implicit synchronisation is not allowed) get the operator application with every temporary --
// the per-face SAT arrays and the device copies of the block/face tables -- placed in
// this file-scope array.  Every GPU that loads the library holds it until the process exits.
constexpr size_t NOALLOC_SCRATCH_BYTES = 8u << 20;   // 8 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {

// device address of g_noalloc_scratch, looked up once per device (host code must not use the
// symbol itself: on the host it is only a stand-in, not a device address)
constexpr int NOALLOC_MAX_DEVICES = 64;
void* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};

int noalloc_scratch(sbp_handle* h, unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return h->fail(SBP_E_CUDA, "cannot query the current device");
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return h->fail(SBP_E_CUDA, std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
        g_noalloc_ptr[dev] = p;
    }
    *out = (unsigned char*)g_noalloc_ptr[dev];
    return SBP_OK;
}

inline size_t align256(size_t x) { return (x + 255) / 256 * 256; }

constexpr int NOALLOC_MAX_BLOCKS = 32;

template <typename T, int O>
void launch_noalloc(sbp_handle* h, const BlockDev* views, int nviews, BlockDev* d_views, FaceRef* d_refs,
                    const StepArgs& a, cudaStream_t st) {
    const int total = h->nface_nodes;
    if (total > 0) k_face_sat<T, O><<<grid_for(total), 256, 0, st>>>(d_views, d_refs, h->nrefs, total, a, h->beta);
    constexpr size_t smem = interior_smem_elems<T, O>() * sizeof(T);
    for (int b = 0; b < nviews; ++b) {
        const BlockDev& v = views[b];
        const int S = v.strip;
        const int ni1 = v.n1 - 2 * S, ni2 = v.n2 - 2 * S;
        dim3 grid((ni1 + ITX - 1) / ITX, (ni2 + ITY - 1) / ITY);
        k_interior<T, O, 1><<<grid, dim3(32, 8), smem, st>>>(v, a);
        const long long nstrip = (long long)v.n1 * v.n2 - (long long)ni1 * ni2;
        k_boundary<T, O, 1><<<grid_for(nstrip), 256, 0, st>>>(v, a);
    }
    if (!h->src_nodes.empty()) {
        const int ns = (int)h->src_nodes.size();
        k_sources<T, 1><<<grid_for(ns), 256, 0, st>>>(d_views, h->d_src_nodes, ns, h->d_src_params, a);
    }
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// misfit gradient: helpers
namespace {

int ensure_adjoint_buffers(sbp_handle* h) {
    bool fresh = false;
    for (auto& hb : h->blocks) {
        if (hb.psi[0]) continue;
        const size_t bytes = 2 * (size_t)hb.n2 * hb.pitch * h->esize;
        hb.psi[0] = h->dalloc(bytes);
        hb.psi[1] = h->dalloc(bytes);
        if (!hb.psi[0] || !hb.psi[1]) return h->fail(SBP_E_OOM, "adjoint fields");
        if (h->precision == SBP_FP32) {
            if (!make_map(&hb.pmaps.u[0], hb.psi[0], hb.pitch, hb.n2, 2, MR, MBOXW) ||
                !make_map(&hb.pmaps.u[1], hb.psi[1], hb.pitch, hb.n2, 2, MR, MBOXW))
                return h->fail(SBP_E_CUDA, "tensor map encoding failed (adjoint fields)");
            hb.pmaps.c = hb.mmaps.c;
        }
        CUtensorMap sm[3];
        if (!make_strip_maps(h, hb, hb.psi[0], hb.psi[1], sm) ||
            cudaMemcpy(hb.d_smaps + 3, sm, sizeof(sm), cudaMemcpyHostToDevice) != cudaSuccess)
            return h->fail(SBP_E_CUDA, "tensor map encoding failed (adjoint strip maps)");
        fresh = true;
    }
    if (!h->d_blocks_adj) {
        h->d_blocks_adj = (BlockDev*)h->dalloc(sizeof(BlockDev) * h->blocks.size());
        if (!h->d_blocks_adj) return h->fail(SBP_E_OOM, "adjoint block views");
        fresh = true;
    }
    return fresh ? sync_views(h) : SBP_OK;
}

// one leapfrog step of the state (the body of sbp_step)
int step_once(sbp_handle* h, double dt, cudaStream_t st) {
    StepArgs a{};
    a.with_data = 1;
    a.dt = dt;
    a.dt2 = dt * dt;
    a.dt2f = (float)a.dt2;
    a.cur = h->cur;
    a.t = h->t;
    fill_basis(h, h->t, a);
    const int rc = run_operator(h, a, 0, st);
    if (rc != SBP_OK) return rc;
    h->cur = 1 - h->cur;
    h->t += dt;
    return SBP_OK;
}

int record_receivers(sbp_handle* h, double* d_row, cudaStream_t st) {
    const int nr = (int)h->recs.size();
    ProfScope ps(h, 6, st, 1);
    if (h->precision == SBP_FP64) k_record<double><<<grid_for(nr, 128), 128, 0, st>>>(h->d_blocks, h->d_recs, nr, h->cur, d_row);
    else k_record<float><<<grid_for(nr, 128), 128, 0, st>>>(h->d_blocks, h->d_recs, nr, h->cur, d_row);
    return SBP_OK;
}

// strip nodes of the gradient (bands of width gs along every face)
long long grad_strip_nodes(const HostBlock& hb, int gs) {
    return (long long)hb.n1 * hb.n2 - (long long)(hb.n1 - 2 * gs) * (hb.n2 - 2 * gs);
}
int order_gs(int o) { return o == 2 ? SBP2_GS : (o == 4 ? SBP4_GS : SBP6_GS); }
// level chunks of the strip gradient: about 4 waves of 256-thread CTAs over the SMs, at most
// one chunk per level and at most GRAD_MAX_CHUNKS
constexpr int GRAD_MAX_CHUNKS = 16;
int grad_strip_chunks(const sbp_handle* h, long long nstrip, int nl) {
    const long long want = 4LL * h->num_sms * 2048;
    long long c = (want + nstrip - 1) / std::max(1LL, nstrip);
    c = std::min<long long>(c, GRAD_MAX_CHUNKS);
    c = std::min<long long>(c, nl);
    return (int)std::max(1LL, c);
}

// gradient contributions of the nl levels of one segment
template <typename T, int O>
void launch_grad(sbp_handle* h, const GradDev* d_grad, const std::vector<GradDev>& grads, int nl, double dt2,
                 cudaStream_t st) {
    const int total = h->nface_nodes;
    if (total > 0) {
        ProfScope ps(h, 6, st, 1);
        k_grad_face<T, O><<<grid_for(total, 128), 128, 0, st>>>(h->d_blocks_adj, d_grad, h->d_refs, h->nrefs, total, nl, h->beta);
    }
    constexpr int GS = GradCfg<O>::GS;
    for (size_t b = 0; b < h->blocks.size(); ++b) {
        const HostBlock& hb = h->blocks[b];
        const BlockDev v = make_view_adj(h, hb);
        {
            ProfScope ps(h, 4, st, 1);
            dim3 gi((hb.n1 - 2 * GS + 31) / 32, (hb.n2 - 2 * GS + 7) / 8);
            k_grad_interior<T, O><<<gi, dim3(32, 8), 0, st>>>(v, grads[b], nl, dt2);
        }
        {
            ProfScope ps(h, 5, st, 2);
            const long long nstrip = grad_strip_nodes(hb, GS);
            const int nchunk = grad_strip_chunks(h, nstrip, nl);
            k_grad_strip<T, O><<<dim3(grid_for(nstrip), nchunk), 256, 0, st>>>(v, grads[b], nl, nchunk, nstrip);
            k_grad_strip_sum<T, O><<<grid_for(nstrip), 256, 0, st>>>(v, grads[b], nchunk, nstrip, dt2);
        }
    }
}

void run_grad(sbp_handle* h, const GradDev* d_grad, const std::vector<GradDev>& grads, int nl, double dt2,
              cudaStream_t st) {
    if (h->precision == SBP_FP64) {
        if (h->order == 2) launch_grad<double, 2>(h, d_grad, grads, nl, dt2, st);
        else if (h->order == 4) launch_grad<double, 4>(h, d_grad, grads, nl, dt2, st);
        else launch_grad<double, 6>(h, d_grad, grads, nl, dt2, st);
    } else {
        if (h->order == 2) launch_grad<float, 2>(h, d_grad, grads, nl, dt2, st);
        else if (h->order == 4) launch_grad<float, 4>(h, d_grad, grads, nl, dt2, st);
        else launch_grad<float, 6>(h, d_grad, grads, nl, dt2, st);
    }
}

// temporaries of one sbp_misfit_gradient call, released on every exit path
struct GradScratch {
    sbp_handle* h;
    std::vector<void*> ptrs;
    explicit GradScratch(sbp_handle* hh) : h(hh) {}
    void* get(size_t bytes) {
        void* p = h->dalloc(bytes);
        if (p) ptrs.push_back(p);
        return p;
    }
    ~GradScratch() {
        cudaDeviceSynchronize();
        for (void* p : ptrs) h->dfree(p);
    }
};

}  // namespace

extern "C" {

const char* sbp_last_error(const sbp_handle* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int sbp_grid_create(const sbp_grid_desc* desc, sbp_handle** out) {
    if (!out) return SBP_E_INVALID_ARG;
    *out = nullptr;
    g_create_error.clear();
    auto bad = [&](int code, const std::string& m) {
        g_create_error = m;
        return code;
    };
    if (!desc) return bad(SBP_E_INVALID_ARG, "null descriptor");
    if (desc->order != 2 && desc->order != 4 && desc->order != 6) return bad(SBP_E_INVALID_ARG, "order must be 2, 4 or 6");
    if (desc->precision != SBP_FP64 && desc->precision != SBP_FP32) return bad(SBP_E_INVALID_ARG, "bad precision");
    if (desc->nblocks < 1 || !desc->blocks) return bad(SBP_E_INVALID_ARG, "need at least one block");
    if (desc->beta < 0 || (desc->beta > 0 && desc->beta < 1)) return bad(SBP_E_INVALID_ARG, "beta must be >= 1");
    if (desc->stencil != SBP_STENCIL_NARROW && desc->stencil != SBP_STENCIL_WIDE) return bad(SBP_E_INVALID_ARG, "bad stencil");
    const int o = desc->order;
    for (int b = 0; b < desc->nblocks; ++b) {
        const sbp_block_desc& bd = desc->blocks[b];
        if (bd.n1 < order_min_n(o) || bd.n2 < order_min_n(o))
            return bad(SBP_E_INVALID_ARG, "block " + std::to_string(b) + ": too few nodes for this order");
        if ((long long)bd.n1 * bd.n2 > (1LL << 31) - 1) return bad(SBP_E_INVALID_ARG, "block too large");
        if (!bd.x1 || !bd.x2) return bad(SBP_E_INVALID_ARG, "null coordinates");
        for (int f = 0; f < 4; ++f) {
            const sbp_face_desc& fd = bd.faces[f];
            if (fd.kind < 0 || fd.kind > 2) return bad(SBP_E_INVALID_ARG, "bad face kind");
            if (fd.kind == SBP_BC_INTERFACE) {
                if (fd.nbr_block < 0 || fd.nbr_block >= desc->nblocks || fd.nbr_face < 0 || fd.nbr_face > 3)
                    return bad(SBP_E_INVALID_ARG, "bad interface neighbour");
                const sbp_block_desc& nb = desc->blocks[fd.nbr_block];
                const sbp_face_desc& back = nb.faces[fd.nbr_face];
                const int nf = f < 2 ? bd.n2 : bd.n1;
                const int nfv = fd.nbr_face < 2 ? nb.n2 : nb.n1;
                const double ht = f < 2 ? (bd.h2 > 0 ? bd.h2 : 1.0 / (bd.n2 - 1)) : (bd.h1 > 0 ? bd.h1 : 1.0 / (bd.n1 - 1));
                const double htv = fd.nbr_face < 2 ? (nb.h2 > 0 ? nb.h2 : 1.0 / (nb.n2 - 1)) : (nb.h1 > 0 ? nb.h1 : 1.0 / (nb.n1 - 1));
                if (nf != nfv || back.kind != SBP_BC_INTERFACE || back.nbr_block != b || back.nbr_face != f ||
                    (back.reversed != 0) != (fd.reversed != 0) || fabs(ht - htv) > 1e-12 * ht || (fd.nbr_block == b && fd.nbr_face == f))
                    return bad(SBP_E_NONCONFORMING_INTERFACE, "interface of block " + std::to_string(b) + " face " +
                                                                  std::to_string(f) + " does not conform");
            }
        }
    }
    sbp_handle* h = new sbp_handle();
    h->order = o;
    h->precision = desc->precision;
    h->esize = desc->precision == SBP_FP64 ? 8 : 4;
    h->beta = desc->beta > 0 ? desc->beta : 1.0;
    h->stencil = desc->stencil;
    h->nblocks = desc->nblocks;
    h->blocks.resize(desc->nblocks);
    auto cleanup = [&](int code, const std::string& m) {
        g_create_error = m;
        sbp_destroy(h);
        return code;
    };
    if (desc->precision == SBP_FP64) { set_smem_attr<double, 2>(); set_smem_attr<double, 4>(); set_smem_attr<double, 6>(); }
    else { set_smem_attr<float, 2>(); set_smem_attr<float, 4>(); set_smem_attr<float, 6>(); }
    h->d_scalar = (double*)h->dalloc(64);
    h->d_flag = (int*)h->dalloc(64);
    h->d_err = (int*)h->dalloc(64);
    if (!h->d_scalar || !h->d_flag || !h->d_err) return cleanup(SBP_E_OOM, "scalar buffers");
    {
        int dev = 0;
        cudaGetDevice(&dev);
        h->device = dev;
        cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (h->num_sms <= 0) h->num_sms = 1;
    }
    {
        int least = 0, greatest = 0;
        cudaDeviceGetStreamPriorityRange(&least, &greatest);
        if (cudaStreamCreateWithPriority(&h->aux, cudaStreamNonBlocking, least) != cudaSuccess ||
            cudaStreamCreateWithPriority(&h->hi, cudaStreamNonBlocking, greatest) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->ev_join_hi, cudaEventDisableTiming) != cudaSuccess)
            return cleanup(SBP_E_CUDA, "auxiliary streams");
    }
    std::vector<FaceRef> refs;
    int start = 0, nintf = 0;
    for (int b = 0; b < desc->nblocks; ++b) {
        const sbp_block_desc& bd = desc->blocks[b];
        HostBlock& hb = h->blocks[b];
        hb.n1 = bd.n1;
        hb.n2 = bd.n2;
        hb.pitch = (bd.n1 + 31) / 32 * 32;
        hb.h1 = bd.h1 > 0 ? bd.h1 : 1.0 / (bd.n1 - 1);
        hb.h2 = bd.h2 > 0 ? bd.h2 : 1.0 / (bd.n2 - 1);
        const size_t plane = (size_t)hb.n2 * hb.pitch;
        const size_t es = h->esize;
        hb.u[0] = h->dalloc(2 * plane * es);
        hb.u[1] = h->dalloc(2 * plane * es);
        if (h->precision == SBP_FP32) {
            hb.du = h->dalloc(2 * plane * es);
            if (!hb.du) return cleanup(SBP_E_OOM, "device allocation failed for block " + std::to_string(b));
        }
        hb.c = h->dalloc(10 * plane * es);
        hb.w = h->dalloc(plane * es);
        hb.r = h->dalloc(2 * plane * es);
        hb.X = (double*)h->dalloc(2 * plane * sizeof(double));
        hb.mx = h->dalloc(closure_elems(o, hb.n2) * es);
        hb.my = h->dalloc(closure_elems(o, hb.n1) * es);
        if (!hb.mx || !hb.my) return cleanup(SBP_E_OOM, "closure matrices");
        hb.G = (double*)h->dalloc(4 * plane * sizeof(double));
        hb.J = (double*)h->dalloc(plane * sizeof(double));
        if (!hb.u[0] || !hb.u[1] || !hb.c || !hb.w || !hb.r || !hb.X || !hb.G || !hb.J)
            return cleanup(SBP_E_OOM, "device allocation failed for block " + std::to_string(b));
        if (h->stencil == SBP_STENCIL_WIDE) {
            hb.gw = h->dalloc(4 * plane * es);
            if (!hb.gw) return cleanup(SBP_E_OOM, "wide-stencil flux planes");
        }
        for (int f = 0; f < 4; ++f) {
            HostFace& F = hb.f[f];
            F.kind = bd.faces[f].kind;
            F.nbr_block = bd.faces[f].nbr_block;
            F.nbr_face = bd.faces[f].nbr_face;
            F.reversed = bd.faces[f].reversed ? 1 : 0;
            F.nf = f < 2 ? hb.n2 : hb.n1;
            F.jhat = (double*)h->dalloc(F.nf * sizeof(double));
            if (!F.jhat) return cleanup(SBP_E_OOM, "face buffers");
            if (h->stencil == SBP_STENCIL_WIDE) {   // SAT terms of the face nodes (k_face_sat)
                F.sat = h->dalloc(4 * (size_t)F.nf * es);
                if (!F.sat) return cleanup(SBP_E_OOM, "face SAT buffers");
            }
            refs.push_back(FaceRef{b, f, start, F.nf});
            start += F.nf;
            if (F.kind == FACE_INTF) {
                F.tr = h->dalloc(7 * (size_t)F.nf * es);
                if (!F.tr) return cleanup(SBP_E_OOM, "interface trace buffers");
                ++nintf;
            }
        }
        if (h->precision == SBP_FP32) {
            if (!make_map(&hb.mmaps.u[0], hb.u[0], hb.pitch, hb.n2, 2, MR, MBOXW) ||
                !make_map(&hb.mmaps.u[1], hb.u[1], hb.pitch, hb.n2, 2, MR, MBOXW) ||
                !make_map(&hb.mmaps.c, hb.c, hb.pitch, hb.n2, 10, MR, MBOXW))
                return cleanup(SBP_E_CUDA, "tensor map encoding failed");
        }
        {
            hb.d_smaps = (CUtensorMap*)h->dalloc(6 * sizeof(CUtensorMap));
            CUtensorMap sm[3];
            if (!hb.d_smaps) return cleanup(SBP_E_OOM, "strip tensor maps");
            if (!make_strip_maps(h, hb, hb.u[0], hb.u[1], sm) ||
                cudaMemcpy(hb.d_smaps, sm, sizeof(sm), cudaMemcpyHostToDevice) != cudaSuccess)
                return cleanup(SBP_E_CUDA, "tensor map encoding failed (strip tiles)");
        }
        // coordinates -> pitched device planes
        double* tmp = (double*)h->staging(2 * (size_t)bd.n1 * bd.n2 * sizeof(double));
        if (!tmp) return cleanup(SBP_E_OOM, "staging buffer");
        const size_t n = (size_t)bd.n1 * bd.n2;
        if (cudaMemcpy(tmp, bd.x1, n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(tmp + n, bd.x2, n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
            return cleanup(SBP_E_CUDA, "coordinate upload failed");
        k_to_pitched<double><<<grid_for(2 * (long long)n), 256>>>(hb.X, tmp, hb.n1, hb.n2, hb.pitch, 2, nullptr);
        const cudaError_t ce = cudaStreamSynchronize(0);
        if (ce != cudaSuccess) return cleanup(SBP_E_CUDA, std::string("coordinate conversion failed: ") + cudaGetErrorString(ce));
    }
    h->nrefs = (int)refs.size();
    h->nface_nodes = start;
    h->d_refs = (FaceRef*)h->dalloc(sizeof(FaceRef) * refs.size());
    h->d_blocks = (BlockDev*)h->dalloc(sizeof(BlockDev) * h->blocks.size());
    if (!h->d_refs || !h->d_blocks) return cleanup(SBP_E_OOM, "tables");
    if (cudaMemcpy(h->d_refs, refs.data(), sizeof(FaceRef) * refs.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return cleanup(SBP_E_CUDA, "face table upload failed");
    h->ntrefs = nintf;
    if (sync_views(h) != SBP_OK) return cleanup(SBP_E_CUDA, h->err);
    {
        // strip tiles (the tile numbering of k_strip_tile: 2 bands of ceil(n1/32) tiles along x1,
        // then 2 side bands of ceil((n2 - 2S)/32) tiles), ordered by a cost estimate: side tiles
        // stage narrow rows, interface tiles read the neighbour, corner tiles carry two faces
        const int S = std::max(order_nclos(o), order_ncol(o));
        std::vector<std::pair<int, int2>> tl;
        for (int b = 0; b < desc->nblocks; ++b) {
            const HostBlock& hb = h->blocks[b];
            const int nbx = (hb.n1 + 31) / 32, nby = (hb.n2 - 2 * S + 31) / 32;
            for (int t = 0; t < 2 * nbx + 2 * nby; ++t) {
                int cost;
                if (t < 2 * nbx) {
                    const int f = 2 + t / nbx, k = t % nbx;
                    cost = (hb.f[f].kind == SBP_BC_INTERFACE ? 3 : 1) + ((k == 0 || k == nbx - 1) ? 2 : 0);
                } else {
                    const int f = (t - 2 * nbx) / nby;
                    cost = 2 + (hb.f[f].kind == SBP_BC_INTERFACE ? 3 : 0);
                }
                tl.push_back({cost, make_int2(b, t)});
            }
        }
        std::stable_sort(tl.begin(), tl.end(),
                         [](const std::pair<int, int2>& x, const std::pair<int, int2>& y) { return x.first > y.first; });
        h->tile_pos.assign(desc->nblocks, {});
        for (int b = 0; b < desc->nblocks; ++b) {
            const HostBlock& hb = h->blocks[b];
            h->tile_pos[b].assign(2 * ((hb.n1 + 31) / 32) + 2 * ((hb.n2 - 2 * S + 31) / 32), -1);
        }
        h->tiles_host.clear();
        for (auto& e : tl) {
            h->tile_pos[e.second.x][e.second.y] = (int)h->tiles_host.size();
            h->tiles_host.push_back(make_int4(e.second.x, e.second.y, 0, 0));
        }
        h->ntiles = (int)h->tiles_host.size();
        h->d_tiles = (int4*)h->dalloc(sizeof(int4) * h->tiles_host.size());
        if (!h->d_tiles) return cleanup(SBP_E_OOM, "tile table");
        if (cudaMemcpy(h->d_tiles, h->tiles_host.data(), sizeof(int4) * h->tiles_host.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return cleanup(SBP_E_CUDA, "tile table upload failed");
    }
    // metric
    cudaMemset(h->d_flag, 0, sizeof(int));
    for (auto& hb : h->blocks) {
        BlockDev b = make_view(h, hb);
        const long long n = (long long)hb.n1 * hb.n2;
        if (o == 2) k_metric<2><<<grid_for(n), 256>>>(b, h->d_flag);
        else if (o == 4) k_metric<4><<<grid_for(n), 256>>>(b, h->d_flag);
        else k_metric<6><<<grid_for(n), 256>>>(b, h->d_flag);
        for (int f = 0; f < 4; ++f) k_face_jhat<<<grid_for(hb.f[f].nf), 256>>>(b, f, hb.f[f].jhat);
    }
    int flag = 0;
    if (cudaMemcpy(&flag, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(0) != cudaSuccess)
        return cleanup(SBP_E_CUDA, "metric setup failed");
    if (flag) return cleanup(SBP_E_JACOBIAN_NONPOSITIVE, "non-positive Jacobian determinant");
    *out = h;
    return SBP_OK;
}

int sbp_destroy(sbp_handle* h) {
    if (!h) return SBP_OK;
    for (void* p : h->allocs)
        if (p) cudaFree(p);
    for (auto& pd : h->pending) {
        cudaEventDestroy(pd.a);
        cudaEventDestroy(pd.b);
    }
    for (auto e : h->ev_pool) cudaEventDestroy(e);
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->aux) cudaStreamDestroy(h->aux);
    if (h->ev_join_hi) cudaEventDestroy(h->ev_join_hi);
    if (h->hi) cudaStreamDestroy(h->hi);
    delete h;
    return SBP_OK;
}

int sbp_set_material(sbp_handle* h, int block, const double* rho, const double* C, int c_layout) {
    if (!h) return SBP_E_INVALID_ARG;
    if (block < 0 || block >= h->nblocks) return h->fail(SBP_E_INVALID_ARG, "bad block index");
    if (!rho || !C) return h->fail(SBP_E_INVALID_ARG, "null material arrays");
    if (c_layout != SBP_C_PAIR10 && c_layout != SBP_C_VOIGT6) return h->fail(SBP_E_INVALID_ARG, "c_layout must be SBP_C_PAIR10 or SBP_C_VOIGT6");
    HostBlock& hb = h->blocks[block];
    const size_t n = (size_t)hb.n1 * hb.n2;
    for (size_t i = 0; i < n; ++i)
        if (!(rho[i] > 0.0) || !std::isfinite(rho[i])) return h->fail(SBP_E_INVALID_ARG, "density must be positive and finite");
    // Voigt input (minor symmetry): every pair entry M[2I+J][2K+L] = C_IJKL is the Voigt entry of
    // its two pair indices (Voigt index 0 for (0,0), 1 for (1,1), 2 for (0,1) and (1,0)); the
    // planes are permuted into the pair layout the material kernel reads
    std::vector<double> expanded;
    if (c_layout == SBP_C_VOIGT6) {
        const int from_voigt[10] = {0, 2, 2, 1, 5, 5, 4, 5, 4, 3};
        expanded.resize(10 * n);
        for (int p = 0; p < 10; ++p) std::memcpy(expanded.data() + p * n, C + from_voigt[p] * n, n * sizeof(double));
        C = expanded.data();
    }
    double* d_rho = (double*)h->staging(11 * n * sizeof(double));
    double* d_C = d_rho ? d_rho + n : nullptr;
    if (!d_rho) return h->fail(SBP_E_OOM, "material staging");
    if (cudaMemcpy(d_rho, rho, n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_C, C, 10 * n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
        return h->fail(SBP_E_CUDA, "material upload failed");
    BlockDev b = make_view(h, hb);
    if (h->precision == SBP_FP64) k_material<double><<<grid_for((long long)n), 256>>>(b, d_rho, d_C);
    else k_material<float><<<grid_for((long long)n), 256>>>(b, d_rho, d_C);
    // the closure rows of D_xx^FC for the new coefficients
    const long long nx = (long long)closure_elems(h->order, hb.n2) / 3, ny = (long long)closure_elems(h->order, hb.n1) / 3;
    if (h->precision == SBP_FP64) {
        if (h->order == 2) { k_closure_mats<double, 2><<<grid_for(nx), 256>>>(b, 0, (double*)hb.mx); k_closure_mats<double, 2><<<grid_for(ny), 256>>>(b, 1, (double*)hb.my); }
        else if (h->order == 4) { k_closure_mats<double, 4><<<grid_for(nx), 256>>>(b, 0, (double*)hb.mx); k_closure_mats<double, 4><<<grid_for(ny), 256>>>(b, 1, (double*)hb.my); }
        else { k_closure_mats<double, 6><<<grid_for(nx), 256>>>(b, 0, (double*)hb.mx); k_closure_mats<double, 6><<<grid_for(ny), 256>>>(b, 1, (double*)hb.my); }
    } else {
        if (h->order == 2) { k_closure_mats<float, 2><<<grid_for(nx), 256>>>(b, 0, (float*)hb.mx); k_closure_mats<float, 2><<<grid_for(ny), 256>>>(b, 1, (float*)hb.my); }
        else if (h->order == 4) { k_closure_mats<float, 4><<<grid_for(nx), 256>>>(b, 0, (float*)hb.mx); k_closure_mats<float, 4><<<grid_for(ny), 256>>>(b, 1, (float*)hb.my); }
        else { k_closure_mats<float, 6><<<grid_for(nx), 256>>>(b, 0, (float*)hb.mx); k_closure_mats<float, 6><<<grid_for(ny), 256>>>(b, 1, (float*)hb.my); }
    }
    cudaError_t e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) return h->fail(SBP_E_CUDA, std::string("material: ") + cudaGetErrorString(e));
    hb.material = true;
    return SBP_OK;
}

int sbp_set_robin(sbp_handle* h, int block, int face, const double* U) {
    if (!h) return SBP_E_INVALID_ARG;
    if (block < 0 || block >= h->nblocks || face < 0 || face > 3 || !U) return h->fail(SBP_E_INVALID_ARG, "bad arguments");
    HostFace& F = h->blocks[block].f[face];
    if (F.kind != SBP_BC_ROBIN) return h->fail(SBP_E_INVALID_ARG, "face is not a Robin face");
    for (int s = 0; s < F.nf; ++s) {
        const double a = U[s], b = U[F.nf + s], c = U[2 * F.nf + s];
        if (!(a >= 0 && c >= 0 && a * c - b * b >= -1e-12 * (a * c + b * b))) return h->fail(SBP_E_INVALID_ARG, "U must be symmetric positive semidefinite");
    }
    if (!F.ju) F.ju = h->dalloc(3 * (size_t)F.nf * h->esize);
    double* tmp = (double*)h->staging(3 * (size_t)F.nf * sizeof(double));
    if (!F.ju || !tmp) return h->fail(SBP_E_OOM, "robin buffers");
    if (cudaMemcpy(tmp, U, 3 * (size_t)F.nf * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
        return h->fail(SBP_E_CUDA, "robin upload failed");
    }
    if (h->precision == SBP_FP64) k_scale_copy<double><<<grid_for(3LL * F.nf), 256>>>((double*)F.ju, tmp, F.jhat, F.nf, 3);
    else k_scale_copy<float><<<grid_for(3LL * F.nf), 256>>>((float*)F.ju, tmp, F.jhat, F.nf, 3);
    cudaError_t e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) return h->fail(SBP_E_CUDA, "robin upload");
    return sync_views(h);
}

int sbp_set_robin_damping(sbp_handle* h, int block, int face, const double* V) {
    if (!h) return SBP_E_INVALID_ARG;
    if (block < 0 || block >= h->nblocks || face < 0 || face > 3 || !V) return h->fail(SBP_E_INVALID_ARG, "bad arguments");
    HostFace& F = h->blocks[block].f[face];
    if (F.kind != SBP_BC_ROBIN) return h->fail(SBP_E_INVALID_ARG, "face is not a Robin face");
    for (int s = 0; s < F.nf; ++s) {
        const double a = V[s], b = V[F.nf + s], c = V[2 * F.nf + s];
        if (!std::isfinite(a) || !std::isfinite(b) || !std::isfinite(c) ||
            !(a >= 0 && c >= 0 && a * c - b * b >= -1e-12 * (a * c + b * b)))
            return h->fail(SBP_E_INVALID_ARG, "V must be symmetric positive semidefinite");
    }
    if (!F.jv) F.jv = h->dalloc(3 * (size_t)F.nf * h->esize);
    double* tmp = (double*)h->staging(3 * (size_t)F.nf * sizeof(double));
    if (!F.jv || !tmp) return h->fail(SBP_E_OOM, "robin damping buffers");
    if (cudaMemcpy(tmp, V, 3 * (size_t)F.nf * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
        return h->fail(SBP_E_CUDA, "robin damping upload failed");
    }
    if (h->precision == SBP_FP64) k_scale_copy<double><<<grid_for(3LL * F.nf), 256>>>((double*)F.jv, tmp, F.jhat, F.nf, 3);
    else k_scale_copy<float><<<grid_for(3LL * F.nf), 256>>>((float*)F.jv, tmp, F.jhat, F.nf, 3);
    cudaError_t e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) return h->fail(SBP_E_CUDA, "robin damping upload");
    h->damping = true;
    if (h->graph_exec) {
        cudaGraphExecDestroy(h->graph_exec);
        h->graph_exec = nullptr;
    }
    return sync_views(h);
}

int sbp_set_layer_dissipation(sbp_handle* h, int block, const double* s) {
    if (!h) return SBP_E_INVALID_ARG;
    if (block < 0 || block >= h->nblocks || !s) return h->fail(SBP_E_INVALID_ARG, "bad arguments");
    HostBlock& hb = h->blocks[block];
    const size_t n = (size_t)hb.n1 * hb.n2;
    for (size_t i = 0; i < n; ++i)
        if (!(s[i] >= 0.0) || !std::isfinite(s[i])) return h->fail(SBP_E_INVALID_ARG, "layer coefficients must be >= 0 and finite");
    // the nodes the dissipation reaches: a centre c with s_c != 0 acts on c-1, c, c+1 along x1 and x2
    std::vector<int2> nodes;
    for (int i2 = 0; i2 < hb.n2; ++i2)
        for (int i1 = 0; i1 < hb.n1; ++i1) {
            bool hit = false;
            for (int o = -1; o <= 1 && !hit; ++o) {
                const int c1 = i1 + o, c2 = i2 + o;
                if (c1 >= 1 && c1 <= hb.n1 - 2 && s[(size_t)i2 * hb.n1 + c1] != 0.0) hit = true;
                if (c2 >= 1 && c2 <= hb.n2 - 2 && s[(size_t)c2 * hb.n1 + i1] != 0.0) hit = true;
            }
            if (hit) nodes.push_back(make_int2(i1, i2));
        }
    const size_t plane = (size_t)hb.n2 * hb.pitch;
    if (!hb.sg) hb.sg = h->dalloc(plane * h->esize);
    h->dfree(hb.d_lnodes);
    h->dfree(hb.lscr);
    hb.d_lnodes = nullptr;
    hb.lscr = nullptr;
    hb.nln = 0;
    double* tmp = (double*)h->staging(n * sizeof(double));
    if (!hb.sg || !tmp) return h->fail(SBP_E_OOM, "layer buffers");
    if (!nodes.empty()) {
        hb.d_lnodes = (int2*)h->dalloc(sizeof(int2) * nodes.size());
        hb.lscr = h->dalloc(2 * nodes.size() * h->esize);
        if (!hb.d_lnodes || !hb.lscr) {
            return h->fail(SBP_E_OOM, "layer buffers");
        }
    }
    if (cudaMemcpy(tmp, s, n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        (!nodes.empty() && cudaMemcpy(hb.d_lnodes, nodes.data(), sizeof(int2) * nodes.size(), cudaMemcpyHostToDevice) != cudaSuccess)) {
        return h->fail(SBP_E_CUDA, "layer upload failed");
    }
    if (h->precision == SBP_FP64) k_to_pitched<double><<<grid_for((long long)n), 256>>>((double*)hb.sg, tmp, hb.n1, hb.n2, hb.pitch, 1, nullptr);
    else k_to_pitched<float><<<grid_for((long long)n), 256>>>((float*)hb.sg, tmp, hb.n1, hb.n2, hb.pitch, 1, nullptr);
    cudaError_t e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) return h->fail(SBP_E_CUDA, "layer upload");
    hb.nln = (int)nodes.size();
    h->layers = false;
    for (auto& b : h->blocks) h->layers = h->layers || b.nln > 0;
    h->damping = h->damping || h->layers;
    if (h->graph_exec) {
        cudaGraphExecDestroy(h->graph_exec);
        h->graph_exec = nullptr;
    }
    return sync_views(h);
}

int sbp_set_time_basis(sbp_handle* h, int nbasis, const int* kinds, const double* omegas) {
    if (!h) return SBP_E_INVALID_ARG;
    if (nbasis < 0 || nbasis > 8 || (nbasis > 0 && (!kinds || !omegas))) return h->fail(SBP_E_INVALID_ARG, "bad time basis");
    for (int k = 0; k < nbasis; ++k)
        if (kinds[k] != 0 && kinds[k] != 1) return h->fail(SBP_E_INVALID_ARG, "basis kind must be 0 (sin) or 1 (cos)");
    if (h->nbasis != 0 && h->nbasis != nbasis) {
        for (auto& hb : h->blocks) {
            if (hb.jf) return h->fail(SBP_E_STATE, "time basis size fixed once data is set");
            for (auto& F : hb.f)
                if (F.g) return h->fail(SBP_E_STATE, "time basis size fixed once data is set");
        }
    }
    h->nbasis = nbasis;
    for (int k = 0; k < nbasis; ++k) {
        h->basis_kind[k] = kinds[k];
        h->basis_omega[k] = omegas[k];
    }
    return SBP_OK;
}

int sbp_set_boundary_data(sbp_handle* h, int block, int face, const double* g) {
    if (!h) return SBP_E_INVALID_ARG;
    if (block < 0 || block >= h->nblocks || face < 0 || face > 3 || !g) return h->fail(SBP_E_INVALID_ARG, "bad arguments");
    if (h->nbasis == 0) return h->fail(SBP_E_STATE, "set the time basis first");
    HostFace& F = h->blocks[block].f[face];
    if (F.kind == SBP_BC_INTERFACE) return h->fail(SBP_E_INVALID_ARG, "interfaces take no boundary data");
    const size_t cnt = 2 * (size_t)h->nbasis * F.nf;
    if (!F.g) F.g = h->dalloc(cnt * h->esize);
    double* tmp = (double*)h->staging(cnt * sizeof(double));
    if (!F.g || !tmp) return h->fail(SBP_E_OOM, "boundary data");
    if (cudaMemcpy(tmp, g, cnt * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
        return h->fail(SBP_E_CUDA, "boundary data upload failed");
    }
    const double* scale = F.kind == SBP_BC_ROBIN ? F.jhat : nullptr;
    if (h->precision == SBP_FP64) k_scale_copy<double><<<grid_for((long long)cnt), 256>>>((double*)F.g, tmp, scale, F.nf, 2 * h->nbasis);
    else k_scale_copy<float><<<grid_for((long long)cnt), 256>>>((float*)F.g, tmp, scale, F.nf, 2 * h->nbasis);
    cudaError_t e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) return h->fail(SBP_E_CUDA, "boundary data upload");
    return sync_views(h);
}

int sbp_set_forcing(sbp_handle* h, int block, const double* f) {
    if (!h) return SBP_E_INVALID_ARG;
    if (block < 0 || block >= h->nblocks || !f) return h->fail(SBP_E_INVALID_ARG, "bad arguments");
    if (h->nbasis == 0) return h->fail(SBP_E_STATE, "set the time basis first");
    HostBlock& hb = h->blocks[block];
    const size_t n = (size_t)hb.n1 * hb.n2, planes = 2 * (size_t)h->nbasis;
    const size_t plane = (size_t)hb.n2 * hb.pitch;
    if (!hb.jf) hb.jf = h->dalloc(planes * plane * h->esize);
    double* tmp = (double*)h->staging(planes * n * sizeof(double));
    if (!hb.jf || !tmp) return h->fail(SBP_E_OOM, "forcing");
    if (cudaMemcpy(tmp, f, planes * n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
        return h->fail(SBP_E_CUDA, "forcing upload failed");
    }
    if (h->precision == SBP_FP64) k_to_pitched<double><<<grid_for((long long)(planes * n)), 256>>>((double*)hb.jf, tmp, hb.n1, hb.n2, hb.pitch, (int)planes, hb.J);
    else k_to_pitched<float><<<grid_for((long long)(planes * n)), 256>>>((float*)hb.jf, tmp, hb.n1, hb.n2, hb.pitch, (int)planes, hb.J);
    cudaError_t e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) return h->fail(SBP_E_CUDA, "forcing upload");
    return sync_views(h);
}

int sbp_add_point_source(sbp_handle* h, int block, double x1, double x2, double f1, double f2, double amplitude,
                         double alpha_p, double t0) {
    if (!h) return SBP_E_INVALID_ARG;
    if (block < 0 || block >= h->nblocks) return h->fail(SBP_E_INVALID_ARG, "bad block");
    if (!(x1 >= 0 && x1 <= 1 && x2 >= 0 && x2 <= 1)) return h->fail(SBP_E_INVALID_ARG, "source outside the block");
    if (!std::isfinite(alpha_p) || !std::isfinite(t0) || !std::isfinite(amplitude)) return h->fail(SBP_E_INVALID_ARG, "non-finite source");
    const HostBlock& hb = h->blocks[block];
    const int q = order_q(h->order);
    auto weights = [&](int N, double hh, double x0, std::vector<int>& nodes, std::vector<double>& w) {
        const double xi = x0 / hh;
        int st = (int)floor(xi) - q + 1;
        st = std::max(0, std::min(st, N - 2 * q));
        for (int i = st; i < st + 2 * q; ++i) nodes.push_back(i);
        for (int i : nodes) {
            double l = 1.0;
            for (int j : nodes)
                if (j != i) l *= (x0 - j * hh) / (i * hh - j * hh);
            w.push_back(l);
        }
    };
    std::vector<int> n1v, n2v;
    std::vector<double> w1, w2;
    weights(hb.n1, hb.h1, x1, n1v, w1);
    weights(hb.n2, hb.h2, x2, n2v, w2);
    const int sid = (int)h->src_params.size();
    h->src_params.push_back(SrcParam{alpha_p, t0});
    for (size_t a = 0; a < n1v.size(); ++a)
        for (size_t c = 0; c < n2v.size(); ++c) {
            const double H = hb.h1 * host_hweight(h->order, hb.n1, n1v[a]) * hb.h2 * host_hweight(h->order, hb.n2, n2v[c]);
            const double wt = amplitude * w1[a] * w2[c] / H;
            SrcNode nd{};
            nd.block = block;
            nd.src = sid;
            nd.gi = (long long)n2v[c] * hb.pitch + n1v[a];
            nd.wt0 = f1 * wt;
            nd.wt1 = f2 * wt;
            h->src_nodes.push_back(nd);
        }
    h->src_dirty = true;
    return upload_sources(h);
}

int sbp_set_state(sbp_handle* h, int block, const double* u_prev, const double* u_cur, double t) {
    if (!h) return SBP_E_INVALID_ARG;
    if (block < 0 || block >= h->nblocks || !u_prev || !u_cur) return h->fail(SBP_E_INVALID_ARG, "bad arguments");
    HostBlock& hb = h->blocks[block];
    const size_t n = (size_t)hb.n1 * hb.n2;
    double* tmp = (double*)h->staging(4 * n * sizeof(double));
    if (!tmp) return h->fail(SBP_E_OOM, "state staging");
    const double* src[2] = {u_prev, u_cur};
    const int dst_idx[2] = {1 - h->cur, h->cur};
    for (int k = 0; k < 2; ++k) {
        double* tk = tmp + 2 * n * k;
        if (cudaMemcpy(tk, src[k], 2 * n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
            return h->fail(SBP_E_CUDA, "state upload failed");
        }
        if (h->precision == SBP_FP64) k_to_pitched<double><<<grid_for(2LL * n), 256>>>((double*)hb.u[dst_idx[k]], tk, hb.n1, hb.n2, hb.pitch, 2, nullptr);
        else k_to_pitched<float><<<grid_for(2LL * n), 256>>>((float*)hb.u[dst_idx[k]], tk, hb.n1, hb.n2, hb.pitch, 2, nullptr);
    }
    // FP32 increment u^n - u^{n-1}: formed from the FP64 levels and rounded once
    if (hb.du) k_diff_to_pitched<<<grid_for(2LL * n), 256>>>((float*)hb.du, tmp + 2 * n, tmp, hb.n1, hb.n2, hb.pitch, 2);
    cudaError_t e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) return h->fail(SBP_E_CUDA, "state upload");
    h->t = t;
    return SBP_OK;
}

namespace {
// device planes of a field of a block (SBP_FIELD_*)
void* field_ptr(const sbp_handle* h, const HostBlock& hb, int which) {
    if (which == SBP_FIELD_APPLY) return hb.r;
    if (which == SBP_FIELD_VELOCITY) return (unsigned char*)hb.rk + 2 * (size_t)hb.n2 * hb.pitch * h->esize;
    return hb.u[which == SBP_FIELD_CUR ? h->cur : 1 - h->cur];
}

// checks of a caller-owned device buffer in the library layout (2 planes of n2 rows x pitch)
int check_device_buffer(sbp_handle* h, const void* p, long long pitch, const HostBlock& hb, const char* what) {
    if (!p) return h->fail(SBP_E_INVALID_ARG, std::string(what) + ": null device pointer");
    if (((uintptr_t)p & 15) != 0) return h->fail(SBP_E_INVALID_ARG, std::string(what) + ": device pointer not 16-byte aligned");
    if (pitch < hb.n1) return h->fail(SBP_E_INVALID_ARG, std::string(what) + ": pitch smaller than n1");
    if ((pitch * (long long)h->esize) % 16 != 0)
        return h->fail(SBP_E_INVALID_ARG, std::string(what) + ": row pitch is not a multiple of 16 bytes");
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess || (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
        cudaGetLastError();
        return h->fail(SBP_E_INVALID_ARG, std::string(what) + ": not a device pointer");
    }
    if (at.type == cudaMemoryTypeDevice && at.device != h->device)
        return h->fail(SBP_E_INVALID_ARG, std::string(what) + ": buffer on another device");
    return SBP_OK;
}
}  // namespace

int sbp_set_state_device(sbp_handle* h, int block, const void* u_prev, const void* u_cur, long long pitch, double t,
                         void* stream) {
    if (!h) return SBP_E_INVALID_ARG;
    if (block < 0 || block >= h->nblocks) return h->fail(SBP_E_INVALID_ARG, "bad block index");
    HostBlock& hb = h->blocks[block];
    int rc = check_device_buffer(h, u_prev, pitch, hb, "u_prev");
    if (rc == SBP_OK) rc = check_device_buffer(h, u_cur, pitch, hb, "u_cur");
    if (rc != SBP_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t es = h->esize;
    // both planes in one pitched copy: plane 1 follows plane 0 after n2 rows on both sides
    const void* src[2] = {u_prev, u_cur};
    void* dst[2] = {hb.u[1 - h->cur], hb.u[h->cur]};
    for (int k = 0; k < 2; ++k)
        if (cudaMemcpy2DAsync(dst[k], hb.pitch * es, src[k], (size_t)pitch * es, hb.n1 * es, 2 * (size_t)hb.n2,
                              cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return h->fail(SBP_E_CUDA, "device state copy failed");
    refresh_increment(h, hb, st);
    h->t = t;
    return check_cuda(h, "device state copy");
}

int sbp_get_field_device(sbp_handle* h, int block, int which, void* dst, long long pitch, void* stream) {
    if (!h) return SBP_E_INVALID_ARG;
    if (block < 0 || block >= h->nblocks || which < 0 || which > 3) return h->fail(SBP_E_INVALID_ARG, "bad arguments");
    HostBlock& hb = h->blocks[block];
    if (which == SBP_FIELD_VELOCITY && !hb.rk) return h->fail(SBP_E_STATE, "no RK4 state on this block");
    int rc = check_device_buffer(h, dst, pitch, hb, "dst");
    if (rc != SBP_OK) return rc;
    const void* src = field_ptr(h, hb, which);
    const size_t es = h->esize;
    if (cudaMemcpy2DAsync(dst, (size_t)pitch * es, src, hb.pitch * es, hb.n1 * es, 2 * (size_t)hb.n2,
                          cudaMemcpyDeviceToDevice, (cudaStream_t)stream) != cudaSuccess)
        return h->fail(SBP_E_CUDA, "device field copy failed");
    return SBP_OK;
}

int sbp_step(sbp_handle* h, int nsteps, double dt, void* stream) {
    if (!h) return SBP_E_INVALID_ARG;
    if (nsteps < 0 || !(dt > 0) || !std::isfinite(dt)) return h->fail(SBP_E_INVALID_ARG, "bad step arguments");
    if (!all_materials(h)) return h->fail(SBP_E_STATE, "set the material of every block first");
    cudaStream_t st = (cudaStream_t)stream;
    StepArgs a{};
    a.with_data = 1;
    a.dt = dt;
    a.dt2 = dt * dt;
    a.dt2f = (float)a.dt2;
    for (int n = 0; n < nsteps; ++n) {
        a.cur = h->cur;
        a.t = h->t;
        fill_basis(h, h->t, a);
        int rc = run_operator(h, a, 0, st);
        if (rc != SBP_OK) return rc;
        h->cur = 1 - h->cur;
        h->t += dt;
    }
    return SBP_OK;
}

int sbp_set_state_rk4(sbp_handle* h, int block, const double* u, const double* v, double t) {
    if (!h) return SBP_E_INVALID_ARG;
    if (block < 0 || block >= h->nblocks || !u || !v) return h->fail(SBP_E_INVALID_ARG, "bad arguments");
    HostBlock& hb = h->blocks[block];
    const size_t n = (size_t)hb.n1 * hb.n2, plane = (size_t)hb.n2 * hb.pitch;
    if (!hb.rk) {
        hb.rk = h->dalloc(10 * plane * h->esize);
        if (!hb.rk) return h->fail(SBP_E_OOM, "RK4 state");
        int rc = sync_views(h);
        if (rc != SBP_OK) return rc;
    }
    double* tmp = (double*)h->staging(2 * n * sizeof(double));
    if (!tmp) return h->fail(SBP_E_OOM, "state staging");
    // u -> RK planes 0-1 and the current state buffer (the first stage input); v -> RK planes 2-3
    void* dst[3] = {hb.rk, hb.u[h->cur], (unsigned char*)hb.rk + 2 * plane * h->esize};
    const double* src[3] = {u, u, v};
    for (int k = 0; k < 3; ++k) {
        if (cudaMemcpy(tmp, src[k], 2 * n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
            return h->fail(SBP_E_CUDA, "state upload failed");
        }
        if (h->precision == SBP_FP64) k_to_pitched<double><<<grid_for(2LL * n), 256>>>((double*)dst[k], tmp, hb.n1, hb.n2, hb.pitch, 2, nullptr);
        else k_to_pitched<float><<<grid_for(2LL * n), 256>>>((float*)dst[k], tmp, hb.n1, hb.n2, hb.pitch, 2, nullptr);
    }
    refresh_increment(h, hb, 0);   // a later leapfrog step continues from the two state buffers
    cudaError_t e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) return h->fail(SBP_E_CUDA, "state upload");
    h->t = t;
    return SBP_OK;
}

int sbp_step_rk4(sbp_handle* h, int nsteps, double dt, void* stream) {
    if (!h) return SBP_E_INVALID_ARG;
    if (nsteps < 0 || !(dt > 0) || !std::isfinite(dt)) return h->fail(SBP_E_INVALID_ARG, "bad step arguments");
    if (!all_materials(h)) return h->fail(SBP_E_STATE, "set the material of every block first");
    for (auto& hb : h->blocks)
        if (!hb.rk) return h->fail(SBP_E_STATE, "set the RK4 state (sbp_set_state_rk4) of every block first");
    cudaStream_t st = (cudaStream_t)stream;
    // the operator-output planes carry the interior point sources of each stage (zero elsewhere)
    for (auto& hb : h->blocks)
        if (cudaMemsetAsync(hb.r, 0, 2 * (size_t)hb.n2 * hb.pitch * h->esize, st) != cudaSuccess)
            return h->fail(SBP_E_CUDA, "RK4 scratch clear failed");
    const double cs[4] = {0.0, 0.5, 0.5, 1.0};
    for (int n = 0; n < nsteps; ++n) {
        for (int s = 1; s <= 4; ++s) {
            StepArgs a{};
            a.with_data = 1;
            a.cur = h->cur;
            a.stage = s;
            a.rkh = dt;
            a.rkhf = (float)dt;
            a.t = h->t + cs[s - 1] * dt;
            fill_basis(h, a.t, a);
            const int rc = run_operator(h, a, 2, st);
            if (rc != SBP_OK) return rc;
            h->cur = 1 - h->cur;
        }
        h->t += dt;
    }
    for (auto& hb : h->blocks) refresh_increment(h, hb, st);
    return check_cuda(h, "RK4 steps");
}

int sbp_apply(sbp_handle* h, int with_data, double t) {
    if (!h) return SBP_E_INVALID_ARG;
    if (!all_materials(h)) return h->fail(SBP_E_STATE, "set the material of every block first");
    StepArgs a{};
    a.cur = h->cur;
    a.with_data = with_data ? 1 : 0;
    a.t = t;
    fill_basis(h, t, a);
    int rc = run_operator(h, a, 1, 0);
    if (rc != SBP_OK) return rc;
    if (cudaDeviceSynchronize() != cudaSuccess) return h->fail(SBP_E_CUDA, "apply failed");
    return check_kernel_errors(h);
}

int sbp_get_field(sbp_handle* h, int block, int which, double* dst) {
    if (!h) return SBP_E_INVALID_ARG;
    if (block < 0 || block >= h->nblocks || !dst || which < 0 || which > 3) return h->fail(SBP_E_INVALID_ARG, "bad arguments");
    HostBlock& hb = h->blocks[block];
    const size_t n = (size_t)hb.n1 * hb.n2;
    if (which == SBP_FIELD_VELOCITY && !hb.rk) return h->fail(SBP_E_STATE, "no RK4 state on this block");
    void* src = field_ptr(h, hb, which);
    double* tmp = (double*)h->staging(2 * n * sizeof(double));
    if (!tmp) return h->fail(SBP_E_OOM, "download staging");
    cudaDeviceSynchronize();
    if (h->precision == SBP_FP64) k_from_pitched<double><<<grid_for(2LL * n), 256>>>(tmp, (const double*)src, hb.n1, hb.n2, hb.pitch, 2);
    else k_from_pitched<float><<<grid_for(2LL * n), 256>>>(tmp, (const float*)src, hb.n1, hb.n2, hb.pitch, 2);
    cudaError_t e = cudaMemcpy(dst, tmp, 2 * n * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return h->fail(SBP_E_CUDA, "download failed");
    return check_kernel_errors(h);
}

int sbp_energy(sbp_handle* h, double dt, double* E_out) {
    if (!h) return SBP_E_INVALID_ARG;
    if (!E_out || !(dt > 0)) return h->fail(SBP_E_INVALID_ARG, "bad arguments");
    if (!all_materials(h)) return h->fail(SBP_E_STATE, "set the material of every block first");
    StepArgs a{};
    a.cur = 1 - h->cur;          // apply A to u^n (the previous level)
    a.with_data = 0;
    int rc = run_operator(h, a, 1, 0);
    if (rc != SBP_OK) return rc;
    cudaMemset(h->d_scalar, 0, sizeof(double));
    for (auto& hb : h->blocks) {
        BlockDev b = make_view(h, hb);
        const int o = h->order;
        const double idt2 = 1.0 / (dt * dt);
        if (h->precision == SBP_FP64) {
            if (o == 2) k_energy<double, 2><<<1024, 256>>>(b, h->cur, idt2, h->d_scalar);
            else if (o == 4) k_energy<double, 4><<<1024, 256>>>(b, h->cur, idt2, h->d_scalar);
            else k_energy<double, 6><<<1024, 256>>>(b, h->cur, idt2, h->d_scalar);
        } else {
            if (o == 2) k_energy<float, 2><<<1024, 256>>>(b, h->cur, idt2, h->d_scalar);
            else if (o == 4) k_energy<float, 4><<<1024, 256>>>(b, h->cur, idt2, h->d_scalar);
            else k_energy<float, 6><<<1024, 256>>>(b, h->cur, idt2, h->d_scalar);
        }
    }
    double E = 0;
    if (cudaMemcpy(&E, h->d_scalar, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return h->fail(SBP_E_CUDA, "energy");
    *E_out = E;
    int rc2 = check_kernel_errors(h);
    if (rc2 != SBP_OK) return rc2;
    if (!std::isfinite(E)) return h->fail(SBP_E_UNSTABLE, "non-finite energy");
    return SBP_OK;
}

int sbp_l2_diff(sbp_handle* h, int which, const double* const* ref, double* err2_out, double* ref2_out) {
    if (!h) return SBP_E_INVALID_ARG;
    if (!ref || which < 0 || which > 3) return h->fail(SBP_E_INVALID_ARG, "bad arguments");
    for (int b = 0; b < h->nblocks; ++b)
        if (!ref[b]) return h->fail(SBP_E_INVALID_ARG, "null reference array");
    for (auto& hb : h->blocks)
        if (which == SBP_FIELD_VELOCITY && !hb.rk) return h->fail(SBP_E_STATE, "no RK4 state");
    if (cudaMemset(h->d_scalar, 0, 2 * sizeof(double)) != cudaSuccess) return h->fail(SBP_E_CUDA, "l2 init");
    for (auto& hb : h->blocks) {
        const size_t n = (size_t)hb.n1 * hb.n2;
        double* tmp = (double*)h->staging(2 * n * sizeof(double));
        if (!tmp) return h->fail(SBP_E_OOM, "l2 staging");
        if (cudaMemcpy(tmp, ref[&hb - h->blocks.data()], 2 * n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
            return h->fail(SBP_E_CUDA, "reference upload failed");
        }
        const BlockDev b = make_view(h, hb);
        const void* U = field_ptr(h, hb, which);
        const int o = h->order;
        if (h->precision == SBP_FP64) {
            if (o == 2) k_l2_diff<double, 2><<<512, 256>>>(b, (const double*)U, tmp, h->d_scalar);
            else if (o == 4) k_l2_diff<double, 4><<<512, 256>>>(b, (const double*)U, tmp, h->d_scalar);
            else k_l2_diff<double, 6><<<512, 256>>>(b, (const double*)U, tmp, h->d_scalar);
        } else {
            if (o == 2) k_l2_diff<float, 2><<<512, 256>>>(b, (const float*)U, tmp, h->d_scalar);
            else if (o == 4) k_l2_diff<float, 4><<<512, 256>>>(b, (const float*)U, tmp, h->d_scalar);
            else k_l2_diff<float, 6><<<512, 256>>>(b, (const float*)U, tmp, h->d_scalar);
        }
        const cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return h->fail(SBP_E_CUDA, std::string("l2 reduction: ") + cudaGetErrorString(e));
    }
    double r[2] = {0, 0};
    if (cudaMemcpy(r, h->d_scalar, sizeof(r), cudaMemcpyDeviceToHost) != cudaSuccess) return h->fail(SBP_E_CUDA, "l2 read");
    if (err2_out) *err2_out = r[0];
    if (ref2_out) *ref2_out = r[1];
    return SBP_OK;
}

int sbp_suggest_dt(sbp_handle* h, double cfl, double* dt_out) {
    if (!h) return SBP_E_INVALID_ARG;
    if (!dt_out || !(cfl > 0)) return h->fail(SBP_E_INVALID_ARG, "bad arguments");
    if (!all_materials(h)) return h->fail(SBP_E_STATE, "set the material of every block first");
    // two passes over every block (the operator-output planes serve as scratch for the per-node
    // FP32 estimates): the FP32 sweep and its minimum, then FP64 refinement near that minimum
    unsigned long long init = 0x7FF0000000000000ULL;   // +inf
    unsigned initf = 0x7F800000u;                       // +inf (FP32)
    unsigned* minf = reinterpret_cast<unsigned*>(h->d_scalar + 1);
    if (cudaMemcpy(h->d_scalar, &init, sizeof(init), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(minf, &initf, sizeof(initf), cudaMemcpyHostToDevice) != cudaSuccess)
        return h->fail(SBP_E_CUDA, "cfl initialisation failed");
    for (int pass = 0; pass < 2; ++pass)
        for (auto& hb : h->blocks) {
            BlockDev b = make_view(h, hb);
            const long long n = (long long)hb.n1 * hb.n2;
            float* rf = reinterpret_cast<float*>(hb.r);
            if (pass == 0) {
                if (h->precision == SBP_FP64) k_cfl_sweep<double><<<grid_for(n), 256>>>(b, rf, minf);
                else k_cfl_sweep<float><<<grid_for(n), 256>>>(b, rf, minf);
            } else {
                if (h->precision == SBP_FP64) k_cfl_refine<double><<<grid_for(n), 256>>>(b, rf, minf, 1e-3f, (unsigned long long*)h->d_scalar);
                else k_cfl_refine<float><<<grid_for(n), 256>>>(b, rf, minf, 1e-3f, (unsigned long long*)h->d_scalar);
            }
        }
    double r = 0;
    if (cudaMemcpy(&r, h->d_scalar, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return h->fail(SBP_E_CUDA, "cfl");
    *dt_out = cfl * r;
    return SBP_OK;
}

int sbp_profile(sbp_handle* h, int enable) {
    if (!h) return SBP_E_INVALID_ARG;
    cudaDeviceSynchronize();
    for (auto& pd : h->pending) {
        h->ev_pool.push_back(pd.a);
        h->ev_pool.push_back(pd.b);
    }
    h->pending.clear();
    for (int k = 0; k < SBP_PROF_FAMILIES; ++k) {
        h->prof_ms[k] = 0;
        h->launches[k] = 0;
    }
    h->prof = enable != 0;
    return SBP_OK;
}

int sbp_profile_read(sbp_handle* h, double* ms, long long* launches) {
    if (!h) return SBP_E_INVALID_ARG;
    for (auto& pd : h->pending) {
        float t = 0;
        if (cudaEventSynchronize(pd.b) != cudaSuccess || cudaEventElapsedTime(&t, pd.a, pd.b) != cudaSuccess)
            return h->fail(SBP_E_CUDA, "event timing failed");
        h->prof_ms[pd.fam] += t;
        h->ev_pool.push_back(pd.a);
        h->ev_pool.push_back(pd.b);
    }
    h->pending.clear();
    for (int k = 0; k < SBP_PROF_FAMILIES; ++k) {
        if (ms) ms[k] = h->prof_ms[k];
        if (launches) launches[k] = h->launches[k];
    }
    return SBP_OK;
}

int sbp_apply_noalloc(sbp_handle* h, const void* u_dev, void* r_dev, int with_data, double t, void* stream) {
    if (!h) return SBP_E_INVALID_ARG;
    if (!u_dev || !r_dev) return h->fail(SBP_E_INVALID_ARG, "null device buffer");
    if (!all_materials(h)) return h->fail(SBP_E_STATE, "set the material of every block first");
    if (h->stencil != SBP_STENCIL_NARROW) return h->fail(SBP_E_STATE, "sbp_apply_noalloc applies the narrow stencil");
    {
        int dev = -1;
        if (cudaGetDevice(&dev) != cudaSuccess || dev != h->device)
            return h->fail(SBP_E_STATE, "sbp_apply_noalloc: the current device is not the device of the handle");
    }
    const int nb = (int)h->blocks.size();
    if (nb > NOALLOC_MAX_BLOCKS) return h->fail(SBP_E_INVALID_ARG, "sbp_apply_noalloc supports at most 32 blocks");
    const size_t es = h->esize;
    // scratch layout: block views | face refs | per face: SAT (4 x nf) array
    size_t need = align256(sizeof(BlockDev) * nb) + align256(sizeof(FaceRef) * h->nrefs);
    for (auto& hb : h->blocks)
        for (auto& F : hb.f) need += align256(4 * (size_t)F.nf * es);
    if (need > NOALLOC_SCRATCH_BYTES)
        return h->fail(SBP_E_INVALID_ARG, "grid needs more scratch than the fixed 8 MiB of sbp_apply_noalloc");
    unsigned char* base = nullptr;
    int rc = noalloc_scratch(h, &base);
    if (rc != SBP_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    size_t off = 0;
    BlockDev* d_views = (BlockDev*)(base + off);
    off += align256(sizeof(BlockDev) * nb);
    FaceRef* d_refs = (FaceRef*)(base + off);
    off += align256(sizeof(FaceRef) * h->nrefs);
    BlockDev views[NOALLOC_MAX_BLOCKS];
    FaceRef refs[4 * NOALLOC_MAX_BLOCKS];
    size_t uoff = 0;
    int start = 0, nr = 0;
    for (int b = 0; b < nb; ++b) {
        const HostBlock& hb = h->blocks[b];
        BlockDev v = make_view(h, hb);
        const size_t planes2 = 2 * (size_t)hb.n2 * hb.pitch * es;
        v.u[0] = (unsigned char*)const_cast<void*>(u_dev) + uoff;   // read as the current level
        v.u[1] = nullptr;
        v.r = (unsigned char*)r_dev + uoff;
        uoff += planes2;
        for (int f = 0; f < 4; ++f) {
            const size_t fb = align256(4 * (size_t)hb.f[f].nf * es);
            v.f[f].sat = base + off;
            v.f[f].tr = nullptr;       // the face SATs read the neighbour directly
            off += fb;
            refs[nr++] = FaceRef{b, f, start, hb.f[f].nf};
            start += hb.f[f].nf;
        }
        views[b] = v;
    }
    if (cudaMemcpyAsync(d_views, views, sizeof(BlockDev) * nb, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_refs, refs, sizeof(FaceRef) * nr, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return h->fail(SBP_E_CUDA, "table upload to the fixed scratch failed");
    StepArgs a{};
    a.cur = 0;
    a.with_data = with_data ? 1 : 0;
    a.t = t;
    fill_basis(h, t, a);
    if (h->precision == SBP_FP64) {
        if (h->order == 2) launch_noalloc<double, 2>(h, views, nb, d_views, d_refs, a, st);
        else if (h->order == 4) launch_noalloc<double, 4>(h, views, nb, d_views, d_refs, a, st);
        else launch_noalloc<double, 6>(h, views, nb, d_views, d_refs, a, st);
    } else {
        if (h->order == 2) launch_noalloc<float, 2>(h, views, nb, d_views, d_refs, a, st);
        else if (h->order == 4) launch_noalloc<float, 4>(h, views, nb, d_views, d_refs, a, st);
        else launch_noalloc<float, 6>(h, views, nb, d_views, d_refs, a, st);
    }
    // the table copies read the stack arrays above: drain the stream before they go away
    if (cudaStreamSynchronize(st) != cudaSuccess) return h->fail(SBP_E_CUDA, "sbp_apply_noalloc kernels failed");
    return check_cuda(h, "sbp_apply_noalloc");
}

int sbp_step_graph(sbp_handle* h, int nsteps, double dt, void* stream) {
    if (!h) return SBP_E_INVALID_ARG;
    if (nsteps <= 0 || (nsteps & 1) || !(dt > 0) || !std::isfinite(dt))
        return h->fail(SBP_E_INVALID_ARG, "sbp_step_graph needs an even positive step count and dt > 0");
    if (!all_materials(h)) return h->fail(SBP_E_STATE, "set the material of every block first");
    if (h->nbasis != 0) return h->fail(SBP_E_STATE, "sbp_step_graph supports point sources only (no time-basis data)");
    cudaStream_t st = (cudaStream_t)stream;
    if (h->d_time_cap < nsteps) {
        h->dfree(h->d_time);
        h->d_time = (double*)h->dalloc(sizeof(double) * nsteps);
        h->d_time_cap = h->d_time ? nsteps : 0;
        if (!h->d_time) return h->fail(SBP_E_OOM, "graph time buffer");
        if (h->graph_exec) {   // the captured launches point at the old buffer
            cudaGraphExecDestroy(h->graph_exec);
            h->graph_exec = nullptr;
        }
    }
    if (!h->graph_exec || h->graph_steps != nsteps || h->graph_dt != dt) {
        if (h->graph_exec) {
            cudaGraphExecDestroy(h->graph_exec);
            h->graph_exec = nullptr;
        }
        // capture on a private stream: the captured launches read the time from d_time and
        // use fixed buffer parities, so the graph can be replayed from any state with the same
        // parity (nsteps is even)
        cudaStream_t cs;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return h->fail(SBP_E_CUDA, "stream");
        const bool prof = h->prof;
        h->prof = false;
        long long saved[SBP_PROF_FAMILIES];
        for (int k = 0; k < SBP_PROF_FAMILIES; ++k) saved[k] = h->launches[k];
        cudaGraph_t g = nullptr;
        int rc = SBP_OK;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = SBP_E_CUDA;
        for (int n = 0; n < nsteps && rc == SBP_OK; ++n) {
            StepArgs a{};
            a.with_data = 1;
            a.dt2 = dt * dt;
    a.dt2f = (float)a.dt2;
            a.cur = (h->cur + n) & 1;
            a.tstep = n;
            a.tdev = h->d_time;
            a.dt = dt;
            rc = run_operator(h, a, 0, cs);
        }
        if (cudaStreamEndCapture(cs, &g) != cudaSuccess || !g) rc = SBP_E_CUDA;
        cudaStreamDestroy(cs);
        h->prof = prof;
        for (int k = 0; k < SBP_PROF_FAMILIES; ++k) h->launches[k] = saved[k];
        if (rc != SBP_OK) {
            if (g) cudaGraphDestroy(g);
            return h->fail(SBP_E_CUDA, "graph capture failed");
        }
        if (cudaGraphInstantiate(&h->graph_exec, g, 0) != cudaSuccess) {
            cudaGraphDestroy(g);
            h->graph_exec = nullptr;
            return h->fail(SBP_E_CUDA, "graph instantiation failed");
        }
        cudaGraphDestroy(g);
        h->graph_steps = nsteps;
        h->graph_dt = dt;
    }
    // the step times, accumulated exactly as sbp_step does (pageable source: staged at call time)
    std::vector<double> times(nsteps);
    double tt = h->t;
    for (int n = 0; n < nsteps; ++n) {
        times[n] = tt;
        tt += dt;
    }
    if (cudaMemcpyAsync(h->d_time, times.data(), sizeof(double) * nsteps, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaGraphLaunch(h->graph_exec, st) != cudaSuccess)
        return h->fail(SBP_E_CUDA, "graph launch failed");
    // launches in the graph, per family (counted as if launched one by one)
    {
        const int nb = (int)h->blocks.size();
        const int nint = h->precision == SBP_FP32 ? (nb + MARCH_MAX_BLOCKS - 1) / MARCH_MAX_BLOCKS : nb;
        h->launches[0] += (long long)nsteps * nint;
        h->launches[1] += (long long)nsteps;
        if (h->n_src_int > 0) h->launches[3] += nsteps;
    }
    h->t = tt;
    return SBP_OK;
}

int sbp_grid_footprint(const sbp_grid_desc* desc, long long* bytes_out) {
    if (!desc || !bytes_out || desc->nblocks < 1 || !desc->blocks) return SBP_E_INVALID_ARG;
    if (desc->precision != SBP_FP64 && desc->precision != SBP_FP32) return SBP_E_INVALID_ARG;
    const long long es = desc->precision == SBP_FP64 ? 8 : 4;
    long long total = 3 * 256;   // scalars
    auto al = [](long long b) { return (b + 255) / 256 * 256; };
    for (int b = 0; b < desc->nblocks; ++b) {
        const sbp_block_desc& bd = desc->blocks[b];
        if (bd.n1 < 2 || bd.n2 < 2) return SBP_E_INVALID_ARG;
        const long long pitch = (bd.n1 + 31) / 32 * 32;
        const long long plane = (long long)bd.n2 * pitch;
        // u (2 x 2), c (10), w (1), r (2) in the field precision, the FP32 leapfrog increment (2);
        // X (2), G (4), J (1) in FP64
        total += al(2 * plane * es) * 2 + al(10 * plane * es) + al(plane * es) + al(2 * plane * es);
        if (desc->precision == SBP_FP32) total += al(2 * plane * es);
        total += al(2 * plane * 8) + al(4 * plane * 8) + al(plane * 8);
        // closure matrices of D_xx^FC along x1 and x2, strip-tile tensor maps
        if (desc->order == 2 || desc->order == 4 || desc->order == 6)
            total += al((long long)closure_elems(desc->order, bd.n2) * es) + al((long long)closure_elems(desc->order, bd.n1) * es);
        total += al(6 * (long long)sizeof(CUtensorMap));
        if (desc->stencil == SBP_STENCIL_WIDE) total += al(4 * plane * es);   // flux planes
        for (int f = 0; f < 4; ++f) {
            const long long nf = f < 2 ? bd.n2 : bd.n1;
            // J^, Robin J^U, boundary data (2 x up to 8 basis functions), interface trace (7)
            total += al(nf * 8) + al(3 * nf * es) + al(2 * 8 * nf * es);
            if (bd.faces[f].kind == SBP_BC_INTERFACE) total += al(7 * nf * es);
            if (desc->stencil == SBP_STENCIL_WIDE) total += al(4 * nf * es);
        }
    }
    total += 4096;   // block views, face tables, source tables
    *bytes_out = total;
    return SBP_OK;
}

int sbp_set_tuning(sbp_handle* h, int rows_per_cta, int overlap) {
    if (!h) return SBP_E_INVALID_ARG;
    if (rows_per_cta < 0) return h->fail(SBP_E_INVALID_ARG, "rows per CTA must be >= 0");
    if (overlap < -1 || overlap > 1) return h->fail(SBP_E_INVALID_ARG, "overlap must be -1, 0 or 1");
    const bool ov = overlap < 0 ? h->overlap : overlap != 0;
    if ((rows_per_cta != h->rows_per_cta || ov != h->overlap) && h->graph_exec) {
        cudaGraphExecDestroy(h->graph_exec);
        h->graph_exec = nullptr;
    }
    h->rows_per_cta = rows_per_cta;
    h->overlap = ov;
    return SBP_OK;
}

int sbp_autotune(sbp_handle* h, int* rows_out, int* overlap_out) {
    if (!h) return SBP_E_INVALID_ARG;
    if (!all_materials(h)) return h->fail(SBP_E_STATE, "set the material of every block first");
    // candidates for the marching kernel's rows per CTA (FP32 only); 0 = heuristic (one wave of
    // 4 CTAs/SM per block); then whether the strips run concurrently with the interior.  Beside
    // fixed heights, heights sized on the whole launch (the interior tiles of every block in one
    // grid): the tallest tiles whose count fits k waves of 4 CTAs/SM (k = 1, 2), and tiles a half
    // band lower, so that the rows left over form a short extra band that finishes in the tail
    std::vector<int> cand{0};
    if (h->precision == SBP_FP32) {
        for (int r : {16, 32, 64, 128, 256}) cand.push_back(r);
        const int S2 = std::max(order_nclos(h->order), order_ncol(h->order));
        int ncx_all = 0, n2i_max = 1;
        for (auto& hb : h->blocks) {
            ncx_all += march_ncx(hb.n1, S2);
            n2i_max = std::max(n2i_max, hb.n2 - 2 * S2);
        }
        for (int k = 1; k <= 2; ++k) {
            const int ny = std::max(1, 4 * h->num_sms * k / std::max(1, ncx_all));
            for (double f : {0.0, 0.5}) {
                const int r = (int)std::ceil(n2i_max / (ny + f));
                if (r >= 16 && std::find(cand.begin(), cand.end(), r) == cand.end()) cand.push_back(r);
            }
        }
    }
    const int ncand = (int)cand.size();
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = 0;
    float best_ms = 1e30f;
    // candidates are timed on leapfrog steps (the launch pattern that matters); the state they
    // overwrite is saved first and put back afterwards
    StepArgs a{};
    a.cur = h->cur;
    a.with_data = 0;
    a.dt2 = 0.0;
    a.dt2f = 0.f;
    // (u^{n-1}, and the FP32 increment, which the timed steps rewrite with its own value)
    std::vector<void*> keep;
    for (auto& hb : h->blocks) {
        const size_t bytes = 2 * (size_t)hb.n2 * hb.pitch * h->esize;
        void* p = h->dalloc(hb.du ? 2 * bytes : bytes);
        if (!p) {
            for (void* q : keep) h->dfree(q);
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return h->fail(SBP_E_OOM, "autotune state copy");
        }
        keep.push_back(p);
        if (cudaMemcpy(p, hb.u[1 - h->cur], bytes, cudaMemcpyDeviceToDevice) != cudaSuccess ||
            (hb.du && cudaMemcpy((unsigned char*)p + bytes, hb.du, bytes, cudaMemcpyDeviceToDevice) != cudaSuccess)) {
            for (void* q : keep) h->dfree(q);
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return h->fail(SBP_E_CUDA, "autotune state copy failed");
        }
    }
    bool restored = true;
    auto put_back = [&]() {
        for (size_t b = 0; b < h->blocks.size(); ++b) {
            const HostBlock& hb = h->blocks[b];
            const size_t bytes = 2 * (size_t)hb.n2 * hb.pitch * h->esize;
            if (cudaMemcpy(hb.u[1 - h->cur], keep[b], bytes, cudaMemcpyDeviceToDevice) != cudaSuccess ||
                (hb.du && cudaMemcpy(hb.du, (unsigned char*)keep[b] + bytes, bytes, cudaMemcpyDeviceToDevice) != cudaSuccess))
                restored = false;
            h->dfree(keep[b]);
        }
    };
    const int saved = h->rows_per_cta;
    const bool saved_ov = h->overlap;
    long long saved_l[SBP_PROF_FAMILIES];
    for (int k = 0; k < SBP_PROF_FAMILIES; ++k) saved_l[k] = h->launches[k];
    auto time_it = [&](float& tot) -> int {
        tot = 0.f;
        for (int rep = 0; rep < 6; ++rep) {
            cudaEventRecord(e0, 0);
            int rc = run_operator(h, a, 0, 0);   // a step without data from the current level
            cudaEventRecord(e1, 0);
            if (rc != SBP_OK) return rc;
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) tot += ms;            // first repetition is a warm-up
        }
        return SBP_OK;
    };
    auto restore = [&](int rc) {
        cudaDeviceSynchronize();
        put_back();
        h->rows_per_cta = saved;
        h->overlap = saved_ov;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return rc;
    };
    h->overlap = false;
    for (int ci = 0; ci < ncand; ++ci) {
        h->rows_per_cta = cand[ci];
        float tot;
        const int rc = time_it(tot);
        if (rc != SBP_OK) return restore(rc);
        if (tot < best_ms) {
            best_ms = tot;
            best = cand[ci];
        }
    }
    h->rows_per_cta = best;
    // strips beside the interior or after it: the two timed alternately at the chosen height (the
    // height's own time is the minimum over the candidates, so it is not compared directly)
    float sum_seq = 0.f, sum_ov = 0.f;
    for (int k = 0; k < 3; ++k) {
        float t;
        h->overlap = false;
        int rc = time_it(t);
        if (rc != SBP_OK) return restore(rc);
        sum_seq += t;
        h->overlap = true;
        rc = time_it(t);
        if (rc != SBP_OK) return restore(rc);
        sum_ov += t;
    }
    const bool best_ov = sum_ov <= sum_seq;
    h->overlap = best_ov;
    cudaDeviceSynchronize();
    put_back();
    for (int k = 0; k < SBP_PROF_FAMILIES; ++k) h->launches[k] = saved_l[k];
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (h->graph_exec) {   // the captured graph used the previous shape
        cudaGraphExecDestroy(h->graph_exec);
        h->graph_exec = nullptr;
    }
    if (!restored) return h->fail(SBP_E_CUDA, "autotune could not restore the state");
    if (rows_out) *rows_out = best;
    if (overlap_out) *overlap_out = best_ov ? 1 : 0;
    return check_kernel_errors(h);
}

int sbp_debug_wait_probe(sbp_handle* h, int polls) {
    if (!h) return SBP_E_INVALID_ARG;
    if (polls < 1 || polls > (1 << 20)) return h->fail(SBP_E_INVALID_ARG, "polls must be in [1, 2^20]");
    k_wait_probe<<<1, 32>>>(polls, h->d_err);
    return check_cuda(h, "wait probe launch");
}

int sbp_check(sbp_handle* h) {
    if (!h) return SBP_E_INVALID_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return h->fail(SBP_E_CUDA, "device error");
    return check_kernel_errors(h);
}

int sbp_get_time(const sbp_handle* h, double* t_out) {
    if (!h || !t_out) return SBP_E_INVALID_ARG;
    *t_out = h->t;
    return SBP_OK;
}

int sbp_get_info(const sbp_handle* h, long long* nodes_out, int* precision_out, int* order_out) {
    if (!h) return SBP_E_INVALID_ARG;
    long long n = 0;
    for (auto& b : h->blocks) n += (long long)b.n1 * b.n2;
    if (nodes_out) *nodes_out = n;
    if (precision_out) *precision_out = h->precision;
    if (order_out) *order_out = h->order;
    return SBP_OK;
}

int sbp_set_receivers(sbp_handle* h, int nrec, const int* rec) {
    if (!h) return SBP_E_INVALID_ARG;
    if (nrec < 0 || (nrec > 0 && !rec)) return h->fail(SBP_E_INVALID_ARG, "bad receiver arguments");
    std::vector<RecDev> v;
    std::vector<std::pair<int, long long>> seen;
    for (int r = 0; r < nrec; ++r) {
        const int b = rec[3 * r], i1 = rec[3 * r + 1], i2 = rec[3 * r + 2];
        if (b < 0 || b >= h->nblocks) return h->fail(SBP_E_INVALID_ARG, "receiver " + std::to_string(r) + ": bad block");
        const HostBlock& hb = h->blocks[b];
        if (i1 < 0 || i1 >= hb.n1 || i2 < 0 || i2 >= hb.n2)
            return h->fail(SBP_E_INVALID_ARG, "receiver " + std::to_string(r) + ": node outside the block");
        RecDev d{};
        d.block = b;
        d.gi = (long long)i2 * hb.pitch + i1;
        d.hinv = 1.0 / (hb.h1 * host_hweight(h->order, hb.n1, i1) * hb.h2 * host_hweight(h->order, hb.n2, i2));
        seen.push_back({b, d.gi});
        v.push_back(d);
    }
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end())
        return h->fail(SBP_E_INVALID_ARG, "receivers must sit on distinct nodes");
    h->dfree(h->d_recs);
    h->d_recs = nullptr;
    h->recs = v;
    if (nrec > 0) {
        h->d_recs = (RecDev*)h->dalloc(sizeof(RecDev) * nrec);
        if (!h->d_recs) return h->fail(SBP_E_OOM, "receiver table");
        if (cudaMemcpy(h->d_recs, v.data(), sizeof(RecDev) * nrec, cudaMemcpyHostToDevice) != cudaSuccess)
            return h->fail(SBP_E_CUDA, "receiver upload");
    }
    return SBP_OK;
}

int sbp_record(sbp_handle* h, int nsteps, double dt, double* traces) {
    if (!h) return SBP_E_INVALID_ARG;
    if (nsteps < 0 || !(dt > 0) || !std::isfinite(dt)) return h->fail(SBP_E_INVALID_ARG, "bad step arguments");
    if (!all_materials(h)) return h->fail(SBP_E_STATE, "set the material of every block first");
    if (h->recs.empty()) return h->fail(SBP_E_STATE, "set the receivers first");
    const size_t per = 2 * h->recs.size();
    GradScratch sc(h);
    double* d_tr = (double*)sc.get(sizeof(double) * per * std::max(nsteps, 1));
    if (!d_tr) return h->fail(SBP_E_OOM, "trace buffer");
    for (int n = 0; n < nsteps; ++n) {
        int rc = step_once(h, dt, 0);
        if (rc != SBP_OK) return rc;
        record_receivers(h, d_tr + (size_t)n * per, 0);
    }
    if (traces && nsteps > 0 &&
        cudaMemcpy(traces, d_tr, sizeof(double) * per * nsteps, cudaMemcpyDeviceToHost) != cudaSuccess)
        return h->fail(SBP_E_CUDA, "trace download");
    int rc = check_cuda(h, "sbp_record");
    return rc != SBP_OK ? rc : check_kernel_errors(h);
}

int sbp_misfit_gradient(sbp_handle* h, int nsteps, double dt, const double* observed, int checkpoint_every,
                        double* misfit, double* const* grad_rho, double* const* grad_C, int c_layout) {
    if (!h) return SBP_E_INVALID_ARG;
    if (nsteps < 1 || !(dt > 0) || !std::isfinite(dt) || !observed || !misfit || checkpoint_every < 0)
        return h->fail(SBP_E_INVALID_ARG, "bad misfit-gradient arguments");
    if (c_layout != SBP_C_PAIR10 && c_layout != SBP_C_VOIGT6) return h->fail(SBP_E_INVALID_ARG, "c_layout must be SBP_C_PAIR10 or SBP_C_VOIGT6");
    const int ncp = c_layout == SBP_C_VOIGT6 ? 6 : 10;
    if (!all_materials(h)) return h->fail(SBP_E_STATE, "set the material of every block first");
    if (h->recs.empty()) return h->fail(SBP_E_STATE, "set the receivers first");
    if (h->stencil != SBP_STENCIL_NARROW) return h->fail(SBP_E_STATE, "the misfit gradient is built for the narrow stencil");
    if (h->damping) return h->fail(SBP_E_STATE, "the misfit gradient is built without the velocity-dependent terms");
    for (auto& hb : h->blocks)
        for (auto& F : hb.f)
            if (F.kind == SBP_BC_DISPLACEMENT && F.g)
                return h->fail(SBP_E_STATE, "displacement faces with boundary data make the data depend on C; not supported");
    int rc = ensure_adjoint_buffers(h);
    if (rc != SBP_OK) return rc;
    // checkpoint interval: given, or (0) every level kept on the device when the forward and
    // adjoint levels of the whole run fit in 60 % of the free memory (no recomputation), else
    // ceil(sqrt(nsteps))
    int K = checkpoint_every > 0 ? std::min(checkpoint_every, nsteps) : 0;
    if (K == 0) {
        size_t lvl_all = 0, freeb = 0, totalb = 0;
        for (auto& hb : h->blocks) lvl_all += 2 * (size_t)hb.n2 * hb.pitch * h->esize;
        if (cudaMemGetInfo(&freeb, &totalb) == cudaSuccess && (double)(2 * (size_t)nsteps + 8) * lvl_all <= 0.6 * (double)freeb)
            K = nsteps;
        else
            K = std::max(1, (int)std::ceil(std::sqrt((double)nsteps)));
    }
    const int nseg = (nsteps + K - 1) / K;
    // one segment: the forward pass stores the levels as it makes them, so none is recomputed
    const bool keep_all = nseg == 1;
    const size_t es = h->esize;
    const size_t per = 2 * h->recs.size();
    const int nb = (int)h->blocks.size();
    GradScratch sc(h);
    std::vector<void*> ck(nb), seg(nb), pseg(nb), fin(nb);
    std::vector<size_t> lvl_bytes(nb);
    // a checkpoint holds (u_{n-1}, u_n) and, for FP32, the leapfrog increment
    const int nck = h->precision == SBP_FP32 ? 3 : 2;
    std::vector<GradDev> grads(nb);
    for (int b = 0; b < nb; ++b) {
        HostBlock& hb = h->blocks[b];
        const size_t plane = (size_t)hb.n2 * hb.pitch;
        lvl_bytes[b] = 2 * plane * es;
        ck[b] = sc.get((size_t)nseg * nck * lvl_bytes[b]);
        seg[b] = sc.get((size_t)(K + 2) * lvl_bytes[b]);
        pseg[b] = sc.get((size_t)K * lvl_bytes[b]);
        fin[b] = sc.get(nck * lvl_bytes[b]);
        GradDev& G = grads[b];
        G.seg = seg[b];
        G.pseg = pseg[b];
        G.lvl_elems = (long long)(2 * plane);
        G.gc = sc.get(10 * plane * es);
        G.grho = sc.get(plane * es);
        for (int f = 0; f < 4; ++f) G.gsat[f] = sc.get(7 * (size_t)hb.f[f].nf * es);
        G.part = sc.get((size_t)GRAD_MAX_CHUNKS * 11 * grad_strip_nodes(hb, order_gs(h->order)) * es);
        if (!ck[b] || !seg[b] || !pseg[b] || !fin[b] || !G.part || !G.gc || !G.grho || !G.gsat[0] || !G.gsat[1] || !G.gsat[2] || !G.gsat[3])
            return h->fail(SBP_E_OOM, "misfit-gradient workspace (checkpoints every " + std::to_string(K) + " steps)");
    }
    GradDev* d_grad = (GradDev*)sc.get(sizeof(GradDev) * nb);
    double* d_tr = (double*)sc.get(sizeof(double) * per * nsteps);
    double* d_obs = (double*)sc.get(sizeof(double) * per * nsteps);
    double* d_res = (double*)sc.get(sizeof(double) * per * nsteps);
    double* d_part = (double*)sc.get(sizeof(double) * nsteps);
    double* d_phi = (double*)sc.get(sizeof(double));
    if (!d_grad || !d_tr || !d_obs || !d_res || !d_part || !d_phi) return h->fail(SBP_E_OOM, "misfit-gradient tables");
    if (cudaMemcpy(d_grad, grads.data(), sizeof(GradDev) * nb, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_obs, observed, sizeof(double) * per * nsteps, cudaMemcpyHostToDevice) != cudaSuccess)
        return h->fail(SBP_E_CUDA, "misfit-gradient table upload failed");
    cudaStream_t st = 0;
    auto copy = [&](void* dst, const void* src, size_t bytes) {
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st) == cudaSuccess;
    };
    auto lvl_ptr = [&](std::vector<void*>& base, int b, size_t l) { return (unsigned char*)base[b] + l * lvl_bytes[b]; };
    // the state (u_{n-1}, u_n[, increment]) of every block to / from slot `slot` of `base`
    auto save_state = [&](std::vector<void*>& base, size_t slot) {
        for (int b = 0; b < nb; ++b) {
            const HostBlock& hb = h->blocks[b];
            if (!copy(lvl_ptr(base, b, nck * slot), hb.u[1 - h->cur], lvl_bytes[b]) ||
                !copy(lvl_ptr(base, b, nck * slot + 1), hb.u[h->cur], lvl_bytes[b]) ||
                (hb.du && !copy(lvl_ptr(base, b, nck * slot + 2), hb.du, lvl_bytes[b])))
                return false;
        }
        return true;
    };
    auto load_state = [&](std::vector<void*>& base, size_t slot) {
        for (int b = 0; b < nb; ++b) {
            const HostBlock& hb = h->blocks[b];
            if (!copy(hb.u[1 - h->cur], lvl_ptr(base, b, nck * slot), lvl_bytes[b]) ||
                !copy(hb.u[h->cur], lvl_ptr(base, b, nck * slot + 1), lvl_bytes[b]) ||
                (hb.du && !copy(hb.du, lvl_ptr(base, b, nck * slot + 2), lvl_bytes[b])))
                return false;
        }
        return true;
    };
    // forward pass: checkpoints (u_{n-1}, u_n) at the start of every segment, receiver traces
    std::vector<double> ck_t(nseg);
    for (int n = 0; n < nsteps; ++n) {
        if (n % K == 0) {
            const int c = n / K;
            if (!save_state(ck, c)) return h->fail(SBP_E_CUDA, "checkpoint copy");
            ck_t[c] = h->t;
            if (keep_all)
                for (int b = 0; b < nb; ++b)
                    if (!copy(lvl_ptr(seg, b, 0), h->blocks[b].u[1 - h->cur], lvl_bytes[b]) ||
                        !copy(lvl_ptr(seg, b, 1), h->blocks[b].u[h->cur], lvl_bytes[b]))
                        return h->fail(SBP_E_CUDA, "level copy");
        }
        rc = step_once(h, dt, st);
        if (rc != SBP_OK) return rc;
        record_receivers(h, d_tr + (size_t)n * per, st);
        if (keep_all)
            for (int b = 0; b < nb; ++b)
                if (!copy(lvl_ptr(seg, b, (size_t)n + 2), h->blocks[b].u[h->cur], lvl_bytes[b]))
                    return h->fail(SBP_E_CUDA, "level copy");
    }
    const int cur_final = h->cur;
    const double t_final = h->t;
    if (!save_state(fin, 0)) return h->fail(SBP_E_CUDA, "final state copy");
    // misfit: 1/2 dt sum (traces - observed)^2
    {
        ProfScope ps(h, 7, st, 2);
        k_residual<<<nsteps, 256, 0, st>>>(d_tr, d_obs, d_res, (int)per, d_part);
        k_sum_scaled<<<1, 256, 0, st>>>(d_part, nsteps, 0.5 * dt, d_phi);
    }
    // backward pass: psi_{N+1} = psi_{N+2} = 0, accumulators zero
    for (int b = 0; b < nb; ++b) {
        HostBlock& hb = h->blocks[b];
        const size_t plane = (size_t)hb.n2 * hb.pitch;
        cudaMemsetAsync(hb.psi[0], 0, lvl_bytes[b], st);
        cudaMemsetAsync(hb.psi[1], 0, lvl_bytes[b], st);
        cudaMemsetAsync(grads[b].gc, 0, 10 * plane * es, st);
        cudaMemsetAsync(grads[b].grho, 0, plane * es, st);
    }
    int pc = 0;
    StepArgs aa{};
    aa.with_data = 0;
    aa.dt2 = dt * dt;
    aa.dt2f = (float)aa.dt2;
    const int nr = (int)h->recs.size();
    for (int s = nseg - 1; s >= 0; --s) {
        const int a0 = s * K, a1 = std::min(a0 + K, nsteps) - 1;   // 0-based steps of the segment
        // recompute the segment's levels u_{a0} .. u_{a1+2} from its checkpoint (one segment: the
        // forward pass kept them)
        if (!keep_all) {
            if (!load_state(ck, s)) return h->fail(SBP_E_CUDA, "checkpoint restore");
            for (int b = 0; b < nb; ++b) {
                if (!copy(lvl_ptr(seg, b, 0), lvl_ptr(ck, b, (size_t)nck * s), lvl_bytes[b]) ||
                    !copy(lvl_ptr(seg, b, 1), lvl_ptr(ck, b, (size_t)nck * s + 1), lvl_bytes[b]))
                    return h->fail(SBP_E_CUDA, "checkpoint restore");
            }
            h->t = ck_t[s];
            for (int q = a0; q <= a1; ++q) {
                rc = step_once(h, dt, st);
                if (rc != SBP_OK) return rc;
                for (int b = 0; b < nb; ++b)
                    if (!copy(lvl_ptr(seg, b, (size_t)(q - a0 + 2)), h->blocks[b].u[h->cur], lvl_bytes[b]))
                        return h->fail(SBP_E_CUDA, "segment copy");
            }
        }
        // adjoint steps n = q + 1 (1-based) from the last step of the segment down to the first
        for (int q = a1; q >= a0; --q) {
            aa.cur = pc;
            rc = run_operator(h, aa, 0, st, true);          // psi_n = 2 psi_{n+1} - psi_{n+2} + dt^2 W L psi_{n+1}
            if (rc != SBP_OK) return rc;
            pc = 1 - pc;
            {
                ProfScope ps(h, 6, st, 1);
                if (h->precision == SBP_FP64)
                    k_inject<double><<<grid_for(nr, 128), 128, 0, st>>>(h->d_blocks_adj, h->d_recs, nr, pc, d_res + (size_t)q * per, dt);
                else
                    k_inject<float><<<grid_for(nr, 128), 128, 0, st>>>(h->d_blocks_adj, h->d_recs, nr, pc, d_res + (size_t)q * per, dt);
            }
            // keep psi_n for the segment's gradient pass
            for (int b = 0; b < nb; ++b)
                if (!copy(lvl_ptr(pseg, b, (size_t)(q - a0)), h->blocks[b].psi[pc], lvl_bytes[b]))
                    return h->fail(SBP_E_CUDA, "adjoint level copy");
        }
        // the gradient terms of the whole segment: psi level l pairs with forward level l + 1
        run_grad(h, d_grad, grads, a1 - a0 + 1, dt * dt, st);
    }
    rc = check_cuda(h, "misfit gradient");
    if (rc != SBP_OK) return rc;
    // outputs: dPhi/dC (pair layout) and dPhi/drho as dense FP64 arrays
    for (int b = 0; b < nb; ++b) {
        HostBlock& hb = h->blocks[b];
        const size_t n = (size_t)hb.n1 * hb.n2;
        double* dC = (double*)sc.get((size_t)ncp * n * sizeof(double));
        double* dR = (double*)sc.get(n * sizeof(double));
        if (!dC || !dR) return h->fail(SBP_E_OOM, "gradient download staging");
        const BlockDev v = make_view(h, hb);
        ProfScope ps(h, 7, st, 1);
        if (h->precision == SBP_FP64)
            k_grad_to_C<double><<<grid_for((long long)n), 256, 0, st>>>(v, (const double*)grads[b].gc, (const double*)grads[b].grho, dC, dR, ncp == 6);
        else
            k_grad_to_C<float><<<grid_for((long long)n), 256, 0, st>>>(v, (const float*)grads[b].gc, (const float*)grads[b].grho, dC, dR, ncp == 6);
        if (grad_C && grad_C[b] && cudaMemcpy(grad_C[b], dC, (size_t)ncp * n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
            return h->fail(SBP_E_CUDA, "gradient download");
        if (grad_rho && grad_rho[b] && cudaMemcpy(grad_rho[b], dR, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
            return h->fail(SBP_E_CUDA, "gradient download");
    }
    // leave the state where the forward pass ended
    h->cur = cur_final;
    h->t = t_final;
    if (!load_state(fin, 0)) return h->fail(SBP_E_CUDA, "final state restore");
    if (cudaMemcpy(misfit, d_phi, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
        return h->fail(SBP_E_CUDA, "misfit download");
    rc = check_cuda(h, "misfit gradient");
    return rc != SBP_OK ? rc : check_kernel_errors(h);
}

// ---------------------------------------------------------------------------------------------
// Batch of resident shots stepped by the persistent tile-queue kernel (k_batch_step).

}  // extern "C"

struct sbp_batch {
    int order = 0, max_shots = 0, rows = 0;
    int num_sms = 1, ctas = 0;
    sbp::BatchHead* d_head = nullptr;
    sbp::BatchShot* d_shots = nullptr;
    sbp::BatchState* d_state = nullptr;
    int4* d_items = nullptr;
    int items_cap = 0;
    int* d_err = nullptr;
    std::vector<sbp_handle*> shot;          // null: free slot
    std::vector<sbp::BatchShot> mirror;     // host copies of the immutable descriptions
    std::vector<sbp::BatchState> pending;   // state of slots admitted since the last launch
    std::vector<char> pending_set;
    std::vector<BatchState> finished;       // device state of slots a poll saw finished (it no longer changes)
    std::vector<char> finished_set;
    std::vector<int> nint, nstrip;          // work items per slot
    bool dirty = false;
    int graph_k = 0;
    cudaGraphExec_t graph = nullptr;
    std::string err;
    int fail(int code, const std::string& m) {
        err = m;
        return code;
    }
};

namespace {

template <int O> void batch_smem_attr() {
    cudaFuncSetAttribute(k_batch_step<O>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem_bytes<O>());
}
template <int O> size_t batch_smem() { return batch_smem_bytes<O>(); }

void batch_launch(sbp_batch* b, cudaStream_t st) {
    if (b->order == 2) k_batch_step<2><<<b->ctas, MTHREADS, batch_smem<2>(), st>>>(b->d_head, b->d_err);
    else if (b->order == 4) k_batch_step<4><<<b->ctas, MTHREADS, batch_smem<4>(), st>>>(b->d_head, b->d_err);
    else k_batch_step<6><<<b->ctas, MTHREADS, batch_smem<6>(), st>>>(b->d_head, b->d_err);
}

int batch_rows_for(const sbp_batch* b, const HostBlock& hb) {
    if (b->rows > 0) return b->rows;
    return 64;
}

// rebuild and upload the work list: interior tiles of every active shot first (the long items),
// then the strip tiles; uploads the state of newly admitted slots; stream-ordered
int batch_sync(sbp_batch* b, cudaStream_t st) {
    if (!b->dirty) return SBP_OK;
    std::vector<int4> items;
    for (int s = 0; s < b->max_shots; ++s)
        if (b->shot[s])
            for (int k = 0; k < b->nint[s]; ++k) items.push_back(make_int4(s, 0, k, 0));
    for (int s = 0; s < b->max_shots; ++s)
        if (b->shot[s])
            for (int k = 0; k < b->nstrip[s]; ++k) items.push_back(make_int4(s, 1, k, 0));
    if ((int)items.size() > b->items_cap) {
        if (b->d_items) cudaFree(b->d_items);
        b->d_items = nullptr;
        b->items_cap = 0;
        const int cap = (int)items.size() * 2;
        if (cudaMalloc(&b->d_items, sizeof(int4) * cap) != cudaSuccess) return b->fail(SBP_E_OOM, "batch work list");
        b->items_cap = cap;
    }
    if (!items.empty() &&
        cudaMemcpyAsync(b->d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return b->fail(SBP_E_CUDA, "batch work list upload");
    for (int s = 0; s < b->max_shots; ++s) {
        if (!b->pending_set[s]) continue;
        if (cudaMemcpyAsync(b->d_shots + s, &b->mirror[s], sizeof(BatchShot), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(b->d_state + s, &b->pending[s], sizeof(BatchState), cudaMemcpyHostToDevice, st) != cudaSuccess)
            return b->fail(SBP_E_CUDA, "batch shot upload");
        b->pending_set[s] = 0;
    }
    BatchHead hd{};
    hd.items = b->d_items;
    hd.nitems = (int)items.size();
    hd.nshots = b->max_shots;
    hd.shots = b->d_shots;
    hd.state = b->d_state;
    hd.next = 0;
    hd.done = 0;
    if (cudaMemcpyAsync(b->d_head, &hd, sizeof(hd), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return b->fail(SBP_E_CUDA, "batch head upload");
    // the host sources above are staged by the copies at call time (pageable memory) except the
    // members of b, which live until the batch is destroyed
    b->dirty = false;
    return SBP_OK;
}

}  // namespace

extern "C" {

int sbp_batch_create(int order, int max_shots, sbp_batch** out) {
    if (!out) return SBP_E_INVALID_ARG;
    *out = nullptr;
    if ((order != 2 && order != 4 && order != 6) || max_shots < 1 || max_shots > 4096) return SBP_E_INVALID_ARG;
    sbp_batch* b = new sbp_batch();
    b->order = order;
    b->max_shots = max_shots;
    b->shot.assign(max_shots, nullptr);
    b->mirror.assign(max_shots, BatchShot{});
    b->pending.assign(max_shots, BatchState{});
    b->pending_set.assign(max_shots, 0);
    b->finished.assign(max_shots, BatchState{});
    b->finished_set.assign(max_shots, 0);
    b->nint.assign(max_shots, 0);
    b->nstrip.assign(max_shots, 0);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (b->num_sms <= 0) b->num_sms = 1;
    if (order == 2) batch_smem_attr<2>();
    else if (order == 4) batch_smem_attr<4>();
    else batch_smem_attr<6>();
    int per_sm = 0;
    if (order == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_step<2>, MTHREADS, batch_smem<2>());
    else if (order == 4) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_step<4>, MTHREADS, batch_smem<4>());
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_step<6>, MTHREADS, batch_smem<6>());
    b->ctas = std::max(1, per_sm) * b->num_sms;      // persistent: every CTA resident at once
    if (cudaMalloc(&b->d_head, sizeof(BatchHead)) != cudaSuccess || cudaMalloc(&b->d_shots, sizeof(BatchShot) * max_shots) != cudaSuccess ||
        cudaMalloc(&b->d_state, sizeof(BatchState) * max_shots) != cudaSuccess || cudaMalloc(&b->d_err, 64) != cudaSuccess) {
        sbp_batch_destroy(b);
        return SBP_E_OOM;
    }
    cudaMemset(b->d_state, 0, sizeof(BatchState) * max_shots);
    cudaMemset(b->d_err, 0, 64);
    BatchHead hd{};
    hd.nshots = max_shots;
    hd.shots = b->d_shots;
    hd.state = b->d_state;
    if (cudaMemcpy(b->d_head, &hd, sizeof(hd), cudaMemcpyHostToDevice) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        sbp_batch_destroy(b);
        return SBP_E_CUDA;
    }
    *out = b;
    return SBP_OK;
}

int sbp_batch_destroy(sbp_batch* b) {
    if (!b) return SBP_OK;
    cudaDeviceSynchronize();
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->d_head) cudaFree(b->d_head);
    if (b->d_shots) cudaFree(b->d_shots);
    if (b->d_state) cudaFree(b->d_state);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_err) cudaFree(b->d_err);
    delete b;
    return SBP_OK;
}

const char* sbp_batch_last_error(const sbp_batch* b) { return b ? b->err.c_str() : ""; }

int sbp_batch_add(sbp_batch* b, sbp_handle* h, int nsteps, double dt, int* slot_out) {
    if (!b || !h || !slot_out) return SBP_E_INVALID_ARG;
    *slot_out = -1;
    if (nsteps < 0 || !(dt > 0) || !std::isfinite(dt)) return b->fail(SBP_E_INVALID_ARG, "bad step arguments");
    if (h->precision != SBP_FP32 || h->order != b->order || h->nblocks != 1 || h->stencil != SBP_STENCIL_NARROW)
        return b->fail(SBP_E_INVALID_ARG, "batch shots are single-block FP32 narrow-stencil handles of the batch's order");
    const HostBlock& hb = h->blocks[0];
    for (auto& F : hb.f)
        if (F.kind == SBP_BC_INTERFACE) return b->fail(SBP_E_INVALID_ARG, "batch shots have no interfaces");
    if (h->nbasis != 0) return b->fail(SBP_E_STATE, "batch shots take point sources only (no time-basis data)");
    if (h->damping) return b->fail(SBP_E_STATE, "batch shots have no velocity-dependent terms");
    if (!hb.material) return b->fail(SBP_E_STATE, "set the material first");
    for (int s = 0; s < b->max_shots; ++s) if (b->shot[s] == h) return b->fail(SBP_E_STATE, "handle already in the batch");
    int slot = -1;
    for (int s = 0; s < b->max_shots && slot < 0; ++s)
        if (!b->shot[s]) slot = s;
    if (slot < 0) return b->fail(SBP_E_STATE, "batch full");
    if (upload_sources(h) != SBP_OK) return b->fail(SBP_E_CUDA, h->err);
    BatchShot& sh = b->mirror[slot];
    sh = BatchShot{};
    sh.maps = hb.mmaps;
    sh.view = make_view(h, hb);
    sh.tiles = h->d_tiles;
    sh.ssrc = h->d_src_strip;
    sh.isrc = h->d_src_int;
    sh.spar = h->d_src_params;
    sh.nisrc = h->n_src_int;
    sh.rows = batch_rows_for(b, hb);
    sh.dt = dt;
    sh.dt2 = dt * dt;
    sh.dt2f = (float)sh.dt2;
    sh.beta = h->beta;
    const int S = sh.view.strip;
    const int n2i = hb.n2 - 2 * S;
    b->nint[slot] = march_ncx(hb.n1, S) * ((n2i + sh.rows - 1) / sh.rows);
    b->nstrip[slot] = h->ntiles;
    b->pending[slot] = BatchState{nsteps, h->cur, h->t};
    b->pending_set[slot] = 1;
    b->finished_set[slot] = 0;
    b->shot[slot] = h;
    b->dirty = true;
    *slot_out = slot;
    return SBP_OK;
}

int sbp_batch_step(sbp_batch* b, int ksteps, void* stream) {
    if (!b) return SBP_E_INVALID_ARG;
    if (ksteps < 1) return b->fail(SBP_E_INVALID_ARG, "ksteps must be >= 1");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = batch_sync(b, st);
    if (rc != SBP_OK) return rc;
    if (!b->graph || b->graph_k != ksteps) {
        if (b->graph) cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        cudaStream_t cs;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return b->fail(SBP_E_CUDA, "stream");
        cudaGraph_t g = nullptr;
        bool okc = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        for (int k = 0; okc && k < ksteps; ++k) batch_launch(b, cs);
        okc = cudaStreamEndCapture(cs, &g) == cudaSuccess && okc && g;
        cudaStreamDestroy(cs);
        if (!okc || cudaGraphInstantiate(&b->graph, g, 0) != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            b->graph = nullptr;
            return b->fail(SBP_E_CUDA, "batch graph capture failed");
        }
        cudaGraphDestroy(g);
        b->graph_k = ksteps;
    }
    if (cudaGraphLaunch(b->graph, st) != cudaSuccess) return b->fail(SBP_E_CUDA, "batch graph launch failed");
    return SBP_OK;
}

int sbp_batch_poll(sbp_batch* b, int* remaining, void* stream) {
    if (!b || !remaining) return SBP_E_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<BatchState> v(b->max_shots);
    int e = 0;
    if (cudaMemcpyAsync(v.data(), b->d_state, sizeof(BatchState) * b->max_shots, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&e, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return b->fail(SBP_E_CUDA, std::string("batch poll: ") + cudaGetErrorString(cudaGetLastError()));
    for (int s = 0; s < b->max_shots; ++s) {
        if (!b->shot[s]) remaining[s] = -1;
        else remaining[s] = b->pending_set[s] ? b->pending[s].remaining : v[s].remaining;
        if (b->shot[s] && !b->pending_set[s] && v[s].remaining <= 0) {
            b->finished[s] = v[s];
            b->finished_set[s] = 1;
        }
    }
    if (e) {
        cudaMemset(b->d_err, 0, sizeof(int));
        return b->fail(SBP_E_TIMEOUT, "a bounded wait in the batch kernel ran out; results of the last steps are invalid");
    }
    return SBP_OK;
}

int sbp_batch_remove(sbp_batch* b, int slot, void* stream) {
    if (!b) return SBP_E_INVALID_ARG;
    if (slot < 0 || slot >= b->max_shots || !b->shot[slot]) return b->fail(SBP_E_INVALID_ARG, "bad slot");
    cudaStream_t st = (cudaStream_t)stream;
    sbp_handle* h = b->shot[slot];
    BatchState cur{};
    if (b->pending_set[slot]) {
        cur = b->pending[slot];
    } else if (b->finished_set[slot]) {
        cur = b->finished[slot];              // finished shots are skipped by later launches: no read needed
    } else if (cudaMemcpyAsync(&cur, b->d_state + slot, sizeof(cur), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
               cudaStreamSynchronize(st) != cudaSuccess) {
        return b->fail(SBP_E_CUDA, "batch state read");
    }
    // hand the state back to the handle: its levels sit in its own buffers with parity cur
    h->cur = cur.cur;
    h->t = cur.t;
    b->shot[slot] = nullptr;
    b->pending[slot] = BatchState{0, 0, 0.0};
    b->pending_set[slot] = 1;               // the slot's device state is cleared at the next launch
    b->finished_set[slot] = 0;
    b->mirror[slot] = BatchShot{};
    b->nint[slot] = b->nstrip[slot] = 0;
    b->dirty = true;
    return SBP_OK;
}

int sbp_batch_autotune(sbp_batch* b, sbp_handle* h, int* rows_out) {
    if (!b || !h) return SBP_E_INVALID_ARG;
    for (int s = 0; s < b->max_shots; ++s)
        if (b->shot[s]) return b->fail(SBP_E_STATE, "autotune an empty batch");
    // the candidates advance h; its two levels, parity and time are restored afterwards
    const HostBlock& hb = h->blocks[0];
    const size_t bytes = 2 * (size_t)hb.n2 * hb.pitch * h->esize;
    void* keep[2] = {nullptr, nullptr};
    if (cudaMalloc(&keep[0], bytes) != cudaSuccess || cudaMalloc(&keep[1], bytes) != cudaSuccess) {
        if (keep[0]) cudaFree(keep[0]);
        return b->fail(SBP_E_OOM, "autotune state copy");
    }
    const int cur0 = h->cur;
    const double t0 = h->t;
    int rc = SBP_OK;
    if (cudaMemcpy(keep[0], hb.u[0], bytes, cudaMemcpyDeviceToDevice) != cudaSuccess ||
        cudaMemcpy(keep[1], hb.u[1], bytes, cudaMemcpyDeviceToDevice) != cudaSuccess)
        rc = b->fail(SBP_E_CUDA, "autotune state copy");
    const int cand[] = {32, 64, 128, 256};
    int best = 64;
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<int> rem(b->max_shots);
    for (int c = 0; c < 4 && rc == SBP_OK; ++c) {
        b->rows = cand[c];
        int slot = -1;
        rc = sbp_batch_add(b, h, 10, 1e-9, &slot);
        if (rc == SBP_OK) rc = sbp_batch_step(b, 2, nullptr);     // warm-up (and the graph capture)
        if (rc == SBP_OK) {
            cudaEventRecord(e0, 0);
            rc = sbp_batch_step(b, 8, nullptr);
            cudaEventRecord(e1, 0);
        }
        if (rc == SBP_OK) rc = sbp_batch_poll(b, rem.data(), nullptr);
        float ms = 0.f;
        if (rc == SBP_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best = cand[c];
        }
        if (slot >= 0) sbp_batch_remove(b, slot, nullptr);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaDeviceSynchronize();
    if (cudaMemcpy(hb.u[0], keep[0], bytes, cudaMemcpyDeviceToDevice) != cudaSuccess ||
        cudaMemcpy(hb.u[1], keep[1], bytes, cudaMemcpyDeviceToDevice) != cudaSuccess)
        rc = rc != SBP_OK ? rc : b->fail(SBP_E_CUDA, "autotune state restore");
    cudaFree(keep[0]);
    cudaFree(keep[1]);
    h->cur = cur0;
    h->t = t0;
    b->rows = best;
    if (rows_out) *rows_out = best;
    return rc;
}

int sbp_batch_set_rows(sbp_batch* b, int rows) {
    if (!b) return SBP_E_INVALID_ARG;
    if (rows < 0) return b->fail(SBP_E_INVALID_ARG, "rows must be >= 0");
    for (int s = 0; s < b->max_shots; ++s)
        if (b->shot[s]) return b->fail(SBP_E_STATE, "set the tile shape while the batch is empty");
    b->rows = rows;
    return SBP_OK;
}

}  // extern "C"
