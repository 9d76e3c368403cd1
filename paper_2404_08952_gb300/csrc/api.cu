// C ABI of the DOLINC stage library (include/dolinc.h).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <chrono>
#include <fstream>
#include <map>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/dolinc.h"
#include "implicit.cuh"
#include "indicator.cuh"
#include "launch.cuh"
#include "mesh.hpp"

using namespace dol;

namespace {

thread_local std::string g_err;

dolinc_status fail(dolinc_status s, const std::string &msg)
{
    g_err = msg;
    return s;
}

// On failure: report, and clear CUDA's last-error state so that it does not resurface
// in a later call's launch check.
#define CU(call)                                                                                          \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) {                                                                          \
            cudaGetLastError();                                                                           \
            return fail(e_ == cudaErrorMemoryAllocation ? DOLINC_ERR_OOM : DOLINC_ERR_CUDA,               \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                              \
        }                                                                                                 \
    } while (0)

PathFns g_paths[N_PATHS];
IndicatorFns g_ind[N_INDICATOR];
BatchFns g_batch[N_BATCH];
std::once_flag g_once;

void init_paths()
{
    std::memset(g_paths, 0, sizeof g_paths);
    std::memset(g_ind, 0, sizeof g_ind);
    std::memset(g_batch, 0, sizeof g_batch);
    register_indicator(g_ind);
    register_batch(g_batch);
    register_paths_d2s(g_paths);
    register_paths_d2e(g_paths);
    register_paths_d3s(g_paths);
    register_paths_d3e(g_paths);
}

size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

namespace dol {
dolinc_status report_error(dolinc_status s, const std::string &msg) { return fail(s, msg); }
}  // namespace dol

// A part of a partitioned mesh: its plan, the device copies of its exchange lists and
// the progress of the step in flight (dolinc_part_step_begin / _continue).
struct PartState {
    PartPlan plan;
    const int32_t *send_dev = nullptr, *recv_dev = nullptr;   // local cell indices
    bool active = false;     // a step is in progress
    int stage = 0;           // its SSP-RK3 stage
    int cur = 0;             // FP64 path: the order-0 record buffer the stage reads
    int order = -1;          // order of the exchange in flight
    double dt = 0;
    double *u = nullptr;
};

struct dolinc_mesh {
    HostMesh h;
    DevMesh d{};
    std::unique_ptr<PartState> part;
    int device = 0;
    std::vector<void *> allocs;
    const uint8_t *flags = nullptr;
    int bv_nv = 0;                     // variables of the boundary values set (0: none yet)
    std::vector<int32_t> bidx_h;       // host copy of DevMesh::bidx
    int max_faces = 0;                 // largest number of slots of a cell
    std::map<std::string, Tune> tuned;  // launch shapes chosen by dolinc_autotune, per scheme
    // per-kernel timing (dolinc_profile_enable)
    bool prof = false;
    struct Rec {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    double prof_ms[DOLINC_KERNEL_COUNT] = {0};
    int64_t prof_n[DOLINC_KERNEL_COUNT] = {0};
    // side stream for the differential passes a stage does not read (see run_diffs_split)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    ~dolinc_mesh()
    {
        for (auto &r : recs) pool.push_back(r.a), pool.push_back(r.b);
        for (auto e : pool) cudaEventDestroy(e);
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(device);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (side) cudaStreamDestroy(side);
        for (void *p : allocs) cudaFree(p);
        cudaSetDevice(cur);
    }
};

struct dolinc_mlp {
    int device = 0;
    float *theta = nullptr, *q = nullptr, *m = nullptr, *v = nullptr, *g = nullptr, *loss = nullptr;
    uint2 *frag = nullptr;
    bool frag_ok = false;
    int step = 0;
    long long cap = 0;
    float *A1 = nullptr, *A2 = nullptr, *A3 = nullptr, *z = nullptr, *dZa = nullptr, *dZb = nullptr;
    void free_scratch()
    {
        for (float *p : {A1, A2, A3, z, dZa, dZb}) cudaFree(p);
        A1 = A2 = A3 = z = dZa = dZb = nullptr;
        cap = 0;
    }
    ~dolinc_mlp()
    {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(device);
        free_scratch();
        for (void *p : {(void *)theta, (void *)q, (void *)m, (void *)v, (void *)g, (void *)loss, (void *)frag}) cudaFree(p);
        cudaSetDevice(cur);
    }
};

struct dolinc_batch {
    dolinc_mesh *arena = nullptr;      // the concatenated meshes
    int n = 0;
    std::vector<int64_t> cell_off;
    const int32_t *cell_mesh = nullptr;
    int block = 256, grid = 0;         // persistent launch shape (0: from occupancy)
    unsigned spin_limit = 1u << 23;    // polls a grid-barrier wait makes before giving up
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;        // private stream the graph is captured on
    std::string gkey;
    ~dolinc_batch()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (cap) cudaStreamDestroy(cap);
        delete arena;
    }
};

namespace {

template <class T> dolinc_status upload(dolinc_mesh *m, const std::vector<T> &v, const T **out)
{
    void *p = nullptr;
    size_t b = v.size() * sizeof(T);
    CU(cudaMalloc(&p, b > 0 ? b : 16));
    m->allocs.push_back(p);
    if (b) CU(cudaMemcpy(p, v.data(), b, cudaMemcpyHostToDevice));
    *out = static_cast<const T *>(p);
    return DOLINC_OK;
}

// scheme helpers ------------------------------------------------------------------------
int needed_order(const dolinc_scheme &s)
{
    int need = s.r > s.k - s.r - 2 ? s.r : s.k - s.r - 2;
    if ((s.limiter == DOLINC_LIMIT_ENO3_ALL || s.limiter == DOLINC_LIMIT_ENO3_FLAGGED ||
         s.limiter == DOLINC_LIMIT_WENO5_ALL || s.limiter == DOLINC_LIMIT_WENO5_FLAGGED) && need < 2)
        need = 2;
    return need < 1 ? 1 : need;
}

dolinc_status check_scheme_shape(const dolinc_mesh *m, const dolinc_scheme *s);

// A compute call: the scheme fits the mesh, and the Dirichlet/Neumann values are set.
dolinc_status check_scheme(const dolinc_mesh *m, const dolinc_scheme *s)
{
    dolinc_status st = check_scheme_shape(m, s);
    if (st) return st;
    if (m->d.n_bv > 0 && m->bv_nv != s->nv)
        return fail(DOLINC_ERR_INVALID_ARG, "the mesh has Dirichlet/Neumann faces: set their values for nv = " +
                                                std::to_string(s->nv) + " with dolinc_set_boundary_values");
    return DOLINC_OK;
}

// The scheme's parameters and their fit to the mesh (sizes, layouts, tuning).
dolinc_status check_scheme_shape(const dolinc_mesh *m, const dolinc_scheme *s)
{
    if (!m || !s) return fail(DOLINC_ERR_INVALID_ARG, "null mesh or scheme");
    if (s->k < 1 || s->r < 0 || s->r >= s->k) return fail(DOLINC_ERR_INVALID_ARG, "bad stencil (k, r)");
    if (s->n_diff < 1 || s->n_diff > MAXN) return fail(DOLINC_ERR_INVALID_ARG, "n_diff must be in 1..4");
    if (needed_order(*s) > s->n_diff)
        return fail(DOLINC_ERR_INVALID_ARG, "stencil (k, r) / limiter needs more differential orders than n_diff");
    if (s->precision < DOLINC_FP64 || s->precision > DOLINC_FP32_BF16)
        return fail(DOLINC_ERR_INVALID_ARG, "unknown precision");
    if (s->limiter < DOLINC_LIMIT_NONE || s->limiter > DOLINC_LIMIT_WENO5_FLAGGED)
        return fail(DOLINC_ERR_INVALID_ARG, "unknown limiter");
    const int dim = m->h.dim;
    if (s->flux == DOLINC_FLUX_UPWIND || s->flux == DOLINC_FLUX_BURGERS) {
        if (s->nv != 1) return fail(DOLINC_ERR_INVALID_ARG, "scalar fluxes need nv = 1");
    } else if (s->flux == DOLINC_FLUX_RUSANOV) {
        if (s->nv != dim + 2) return fail(DOLINC_ERR_INVALID_ARG, "Euler needs nv = dim + 2");
        if (!(s->gamma > 1.0)) return fail(DOLINC_ERR_INVALID_ARG, "gamma must exceed 1");
    } else {
        return fail(DOLINC_ERR_INVALID_ARG, "unknown flux");
    }
    if ((s->limiter == DOLINC_LIMIT_ENO3_FLAGGED || s->limiter == DOLINC_LIMIT_FIRST_ORDER_FLAGGED ||
         s->limiter == DOLINC_LIMIT_WENO5_FLAGGED) && !m->flags)
        return fail(DOLINC_ERR_INVALID_ARG, "flagged limiter without flags (dolinc_set_flags)");
    return DOLINC_OK;
}

int elem_bytes(int prec, int m) { return prec == DOLINC_FP64 ? 8 : (prec == DOLINC_FP32_BF16 && m >= 2 ? 2 : 4); }
int ncoef_h(int dim, int m) { return dim == 2 ? m + 1 : (m + 1) * (m + 2) / 2; }
int stride_h(int dim, int nv, int m, int prec) { return rec_stride(nv * ncoef_h(dim, m), elem_bytes(prec, m)); }

struct WsLayout {
    size_t status, o0[3], ord[MAXN + 1], ord1b, ustage, dacc, flux, hsend, hrecv, total;
};

// The paired schedule applies: one order above the stencil's (n_diff = 2, order 1 read).
bool pair_scheme(const dolinc_scheme *s) { return s->n_diff == 2 && needed_order(*s) == 1; }

WsLayout ws_layout(const dolinc_mesh *m, const dolinc_scheme *s)
{
    WsLayout L{};
    const size_t nc = (size_t)m->h.n_cells;
    size_t o = 0;
    L.status = o;
    o += 1024;                                  // status word, then the batch grid-barrier words
    // order-0 records: step start and two stage inputs (the third only for the
    // increment form of bulk precisions below FP64)
    const int n_o0 = s->precision == DOLINC_FP64 ? 2 : 3;
    for (int i = 0; i < 3; ++i) {
        L.o0[i] = o;
        if (i < n_o0) o += al256(nc * stride_h(m->h.dim, s->nv, 0, s->precision) * elem_bytes(s->precision, 0));
    }
    L.ord[0] = L.o0[0];
    for (int mm = 1; mm <= MAXN; ++mm) {
        L.ord[mm] = o;
        if (mm <= s->n_diff) o += al256(nc * stride_h(m->h.dim, s->nv, mm, s->precision) * elem_bytes(s->precision, mm));
    }
    L.ord1b = o;                                // second order-1 buffer of the paired schedule
    if (pair_scheme(s)) o += al256(nc * stride_h(m->h.dim, s->nv, 1, s->precision) * elem_bytes(s->precision, 1));
    L.ustage = o;
    o += al256(nc * s->nv * sizeof(double));
    L.dacc = o;                                 // increment accumulator (bulk precision below FP64)
    if (s->precision != DOLINC_FP64) o += al256(nc * s->nv * sizeof(float));
    L.flux = o;                                 // per-face fluxes of the face-centric stage
    o += al256((size_t)m->h.n_faces * s->nv * (s->precision == DOLINC_FP64 ? sizeof(double) : sizeof(float)));
    // part meshes: the halo exchange buffers, sized for the largest record exchanged
    L.hsend = L.hrecv = o;
    if (m->part) {
        size_t rb = 0;
        for (int mm = 0; mm <= s->n_diff; ++mm)
            rb = std::max(rb, (size_t)stride_h(m->h.dim, s->nv, mm, s->precision) * elem_bytes(s->precision, mm));
        o += al256(rb * m->part->plan.send_cells.size());
        L.hrecv = o;
        o += al256(rb * m->part->plan.recv_cells.size());
    }
    L.total = o;
    return L;
}

dolinc_status check_ws(const dolinc_mesh *m, const dolinc_scheme *s, const void *ws, size_t bytes, WsLayout &L)
{
    L = ws_layout(m, s);
    if (!ws) return fail(DOLINC_ERR_INVALID_ARG, "null workspace");
    if (((uintptr_t)ws & 255) != 0) return fail(DOLINC_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (bytes < L.total) return fail(DOLINC_ERR_INVALID_ARG, "workspace too small (see dolinc_workspace_size)");
    return DOLINC_OK;
}

const PathFns *path_for(const dolinc_mesh *m, const dolinc_scheme *s, int ns)
{
    std::call_once(g_once, init_paths);
    const PathFns *p = &g_paths[path_index(m->h.dim, s->nv, ns, s->precision)];
    return p->stage ? p : nullptr;
}

char *B(void *p, size_t off) { return static_cast<char *>(p) + off; }

StageArgs base_args(const dolinc_mesh *m, const dolinc_scheme *s, void *ws, const WsLayout &L, size_t o0off)
{
    StageArgs a{};
    a.ord[0] = B(ws, o0off);
    for (int mm = 1; mm <= MAXN; ++mm) a.ord[mm] = B(ws, L.ord[mm]);
    a.status = reinterpret_cast<unsigned *>(B(ws, L.status));
    a.k = s->k;
    a.r = s->r;
    a.flux = s->flux;
    a.gamma = s->gamma;
    for (int i = 0; i < 3; ++i) a.adv[i] = s->adv[i];
    const bool flagged = s->limiter == DOLINC_LIMIT_ENO3_FLAGGED || s->limiter == DOLINC_LIMIT_FIRST_ORDER_FLAGGED ||
                         s->limiter == DOLINC_LIMIT_WENO5_FLAGGED;
    a.flags = flagged ? m->flags : nullptr;
    a.all_mode = s->limiter == DOLINC_LIMIT_ENO3_ALL ? LIM_ENO3 : s->limiter == DOLINC_LIMIT_WENO5_ALL ? LIM_WENO5 : LIM_NONE;
    a.flag_mode = s->limiter == DOLINC_LIMIT_FIRST_ORDER_FLAGGED ? LIM_FIRST_ORDER
                : s->limiter == DOLINC_LIMIT_WENO5_FLAGGED       ? LIM_WENO5
                                                                 : LIM_ENO3;
    a.face_flux = B(ws, L.flux);
    return a;
}

cudaEvent_t take_event(dolinc_mesh *m)
{
    if (!m->pool.empty()) {
        cudaEvent_t e = m->pool.back();
        m->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Runs `launch` bracketed by events when profiling is on.
template <class F> void timed(dolinc_mesh *m, int kind, cudaStream_t s, F &&launch)
{
    if (!m->prof) {
        launch();
        return;
    }
    dolinc_mesh::Rec r{kind, take_event(m), take_event(m)};
    cudaEventRecord(r.a, s);
    launch();
    cudaEventRecord(r.b, s);
    m->recs.push_back(r);
}

std::string scheme_key(const dolinc_mesh *m, const dolinc_scheme *s)
{
    std::ostringstream k;
    k << m->h.dim << "d_nv" << s->nv << "_ns" << needed_order(*s) << "_nd" << s->n_diff << "_p" << s->precision
      << "_c" << m->h.n_cells << "_f" << m->h.n_faces << "_mf" << m->max_faces;
    return k.str();
}

Tune tune_for(const dolinc_mesh *m, const dolinc_scheme *s)
{
    auto it = m->tuned.find(scheme_key(m, s));
    if (it != m->tuned.end()) return it->second;
    Tune t;                                       // heuristic: one lane per face slot
    t.diff_lpc = t.stage_lpc = m->max_faces <= 4 ? 4 : 8;
    return t;
}

// differential passes 1..n from the order-0 record at o0off
void run_diffs(dolinc_mesh *m, const PathFns *p, void *ws, const WsLayout &L, size_t o0off, int n,
               const Tune &t, cudaStream_t st)
{
    for (int mm = 1; mm <= n; ++mm)
        timed(m, mm, st, [&] {
            p->diff(m->d, mm, B(ws, mm == 1 ? o0off : L.ord[mm - 1]), B(ws, L.ord[mm]), t,
                    reinterpret_cast<unsigned *>(B(ws, L.status)), st);
            if (mm == 1) p->bnd_grad(m->d, B(ws, o0off), B(ws, L.ord[1]), st);
        });
}

// Differential passes of one stage.  The passes the stencil reads (through
// needed_order) run on `st`; the higher orders the scheme also computes are read by
// nothing in the stage, so they run on the mesh's side stream, overlapping the stage.
// Returns true when the side stream holds work the caller must join (m->ev_join)
// before the next pass rewrites the records those passes read.
bool run_diffs_split(dolinc_mesh *m, const PathFns *p, void *ws, const WsLayout &L, size_t o0off,
                     const dolinc_scheme *s, const Tune &t, cudaStream_t st)
{
    const int need = needed_order(*s);
    if (s->n_diff > need && !m->side) {
        if (cudaStreamCreateWithFlags(&m->side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&m->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&m->ev_join, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            if (m->side) cudaStreamDestroy(m->side);
            if (m->ev_fork) cudaEventDestroy(m->ev_fork);
            m->side = nullptr;
            m->ev_fork = m->ev_join = nullptr;
        }
    }
    if (s->n_diff <= need || !m->side) {
        run_diffs(m, p, ws, L, o0off, s->n_diff, t, st);
        return false;
    }
    run_diffs(m, p, ws, L, o0off, need, t, st);
    cudaEventRecord(m->ev_fork, st);
    cudaStreamWaitEvent(m->side, m->ev_fork, 0);
    for (int mm = need + 1; mm <= s->n_diff; ++mm)
        timed(m, mm, m->side, [&] {
            p->diff(m->d, mm, B(ws, L.ord[mm - 1]), B(ws, L.ord[mm]), t, reinterpret_cast<unsigned *>(B(ws, L.status)),
                    m->side);
        });
    cudaEventRecord(m->ev_join, m->side);
    return true;
}

dolinc_status launch_check()
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(DOLINC_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return DOLINC_OK;
}

}  // namespace

dolinc_status upload_mesh(dolinc_mesh *m);

extern "C" {

const char *dolinc_last_error(void) { return g_err.c_str(); }

dolinc_status dolinc_mesh_create(const dolinc_mesh_desc *desc, dolinc_mesh **out)
{
    if (!out) return fail(DOLINC_ERR_INVALID_ARG, "null output handle");
    *out = nullptr;
    if (!desc) return fail(DOLINC_ERR_INVALID_ARG, "null descriptor");
    dolinc_mesh *m = new (std::nothrow) dolinc_mesh();
    if (!m) return fail(DOLINC_ERR_OOM, "host allocation");
    std::string err;
    try {
        err = build_host_mesh(*desc, m->h);
    } catch (const std::bad_alloc &) {
        delete m;
        return fail(DOLINC_ERR_OOM, "host allocation while building the mesh");
    }
    if (!err.empty()) {
        delete m;
        return fail(DOLINC_ERR_MESH, err);
    }
    dolinc_status st = upload_mesh(m);
    if (st) {
        delete m;
        return st;
    }
    *out = m;
    return DOLINC_OK;
}

}  // extern "C"

// Gauss weight tables of the differential passes: per slot ((1-w_c) S / V_c, the
// neighbour id bits), per cell (sum w_c S / V_c, 1 / V_c), FP64 and FP32.
void weight_tables(const HostMesh &h, std::vector<double> &sk64, std::vector<float> &sk32, std::vector<double> &ck64,
                   std::vector<float> &ck32)
{
    const int64_t nc = h.n_cells, ns = h.n_slots;
    sk64.assign(4 * ns, 0.0);
    sk32.assign(4 * ns, 0.0f);
    ck64.assign(4 * nc, 0.0);
    ck32.assign(4 * nc, 0.0f);
    for (int64_t s = 0; s < ns; ++s) {
        for (int k = 0; k < 3; ++k) {
            sk64[4 * s + k] = h.ss[3 * s + k];
            sk32[4 * s + k] = (float)h.ss[3 * s + k];
        }
        long long nbits = (long long)h.snb[s];
        std::memcpy(&sk64[4 * s + 3], &nbits, 8);
        int ib = h.snb[s];
        std::memcpy(&sk32[4 * s + 3], &ib, 4);
    }
    for (int64_t c = 0; c < nc; ++c)
        for (int k = 0; k < 4; ++k) {
            ck64[4 * c + k] = h.cw[4 * c + k];
            ck32[4 * c + k] = (float)h.cw[4 * c + k];
        }
}

// Copies the host tables of m->h to the device (FP64 and FP32 derived tables).
dolinc_status upload_mesh(dolinc_mesh *m)
{
    cudaGetDevice(&m->device);
    const HostMesh &h = m->h;
    const int64_t nc = h.n_cells, nf = h.n_faces, ns = h.n_slots;
    std::vector<int2> slot2(ns + 2, make_int2(0, 0));   // two spare entries: bulk copies round to 16 bytes
    std::vector<double> sk64, ck64, f64(8 * nf);
    std::vector<float> sk32, ck32, f32(8 * nf);
    for (int64_t s = 0; s < ns; ++s) slot2[s] = make_int2(h.snb[s], (int)h.sword[s]);
    std::vector<uint32_t> sword(h.sword.begin(), h.sword.end());
    sword.resize(ns + 4, 0u);                           // spare entries: 16-byte loads of 4 words
    weight_tables(h, sk64, sk32, ck64, ck32);
    std::vector<int32_t> fo(nf), fn(nf), fe(nf);
    std::vector<int8_t> ff(nf);
    for (int64_t f = 0; f < nf; ++f) {
        double r[8] = {h.fd[3 * f], h.fd[3 * f + 1], h.fd[3 * f + 2], h.fg[f],
                       h.fS[3 * f], h.fS[3 * f + 1], h.fS[3 * f + 2], 0.0};
        r[7] = std::sqrt(r[4] * r[4] + r[5] * r[5] + r[6] * r[6]);
        for (int k = 0; k < 8; ++k) {
            f64[8 * f + k] = r[k];
            f32[8 * f + k] = (float)r[k];
        }
        fo[f] = (int32_t)h.fo[f];
        fn[f] = (int32_t)h.fn[f];
        fe[f] = (int32_t)h.face_ext[f];
        ff[f] = h.face_flip[f];
    }
    std::vector<int32_t> off(h.off.begin(), h.off.end());
    m->max_faces = 0;
    for (int64_t c = 0; c < nc; ++c) m->max_faces = std::max(m->max_faces, (int)(h.off[c + 1] - h.off[c]));
    // first internal face owned by each cell (faces are sorted by owner)
    std::vector<int32_t> fown(nc + 1, 0);
    for (int64_t f = 0; f < nf; ++f) fown[h.fo[f] + 1]++;
    for (int64_t c = 0; c < nc; ++c) fown[c + 1] += fown[c];
    int mtf[3] = {0, 0, 0};
    const int tiles[3] = {64, 128, 256};
    for (int ti = 0; ti < 3; ++ti)
        for (int64_t t0 = 0; t0 < nc; t0 += tiles[ti]) {
            int64_t t1 = std::min<int64_t>(nc, t0 + tiles[ti]);
            mtf[ti] = std::max(mtf[ti], fown[t1] - fown[t0]);
        }
    dolinc_status st = DOLINC_OK;
    DevMesh &d = m->d;
    d.dim = h.dim;
    d.n_cells = (int)nc;
    d.n_faces = (int)nf;
    d.n_slots = (int)ns;
    for (int ti = 0; ti < 3; ++ti) d.max_tile_faces[ti] = mtf[ti];
    d.max_slots = m->max_faces;
    d.uniform_slots = m->max_faces;
    for (int64_t c = 0; c < nc; ++c)
        if (h.off[c + 1] - h.off[c] != m->max_faces) {
            d.uniform_slots = 0;
            break;
        }
    // Dirichlet / Neumann faces: index, kind, normal distance, and the cells holding them
    std::vector<int32_t> bidx(nf, -1), bcell, bcell_off(1, 0), bcell_face;
    std::vector<int8_t> bkind;
    std::vector<double> bdelta64;
    std::vector<float> bdelta32;
    for (int64_t f = 0; f < nf && !h.fkind.empty(); ++f) {
        if (h.fkind[f] < 2) continue;
        bidx[f] = (int32_t)bkind.size();
        bkind.push_back(h.fkind[f]);
        const double *S = &h.fS[3 * f], *xf = &h.fxf[3 * f], *xc = &h.xc[3 * h.fo[f]];
        const double sn = std::sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
        const double dl = ((xf[0] - xc[0]) * S[0] + (xf[1] - xc[1]) * S[1] + (xf[2] - xc[2]) * S[2]) / sn;
        bdelta64.push_back(dl);
        bdelta32.push_back((float)dl);
    }
    // faces are sorted by owner, so a cell's boundary faces are consecutive
    for (int64_t f = 0; f < nf; ++f) {
        if (bidx[f] < 0) continue;
        if (bcell.empty() || bcell.back() != (int32_t)h.fo[f]) {
            if (!bcell.empty()) bcell_off.push_back((int32_t)bcell_face.size());
            bcell.push_back((int32_t)h.fo[f]);
        }
        bcell_face.push_back((int32_t)f);
    }
    if (!bcell.empty()) bcell_off.push_back((int32_t)bcell_face.size());
    m->bidx_h = bidx;
    d.n_bv = (int)bkind.size();
    d.n_bcell = (int)bcell.size();
    d.bval64 = nullptr;
    d.bval32 = nullptr;
    if (d.n_bv > 0) {
        if ((st = upload(m, bidx, &d.bidx)) || (st = upload(m, bkind, &d.bkind)) ||
            (st = upload(m, bdelta64, &d.bdelta64)) || (st = upload(m, bdelta32, &d.bdelta32)) ||
            (st = upload(m, bcell, &d.bcell)) || (st = upload(m, bcell_off, &d.bcell_off)) ||
            (st = upload(m, bcell_face, &d.bcell_face)))
            return st;
    } else {
        d.bidx = nullptr;
    }
    if ((st = upload(m, off, &d.off)) || (st = upload(m, slot2, &d.slot2)) || (st = upload(m, sword, &d.sword)) ||
        (st = upload(m, sk64, &d.slotk64)) ||
        (st = upload(m, sk32, &d.slotk32)) || (st = upload(m, ck64, &d.cellk64)) ||
        (st = upload(m, ck32, &d.cellk32)) || (st = upload(m, f64, &d.face64)) || (st = upload(m, f32, &d.face32)) ||
        (st = upload(m, fo, &d.fo)) || (st = upload(m, fn, &d.fn)) || (st = upload(m, fe, &d.face_ext)) ||
        (st = upload(m, ff, &d.face_flip)) || (st = upload(m, fown, &d.fown)))
        return st;
    return DOLINC_OK;
}

extern "C" {

void dolinc_mesh_destroy(dolinc_mesh *mesh) { delete mesh; }

dolinc_status dolinc_mesh_get_info(const dolinc_mesh *m, dolinc_mesh_info *info)
{
    if (!m || !info) return fail(DOLINC_ERR_INVALID_ARG, "null argument");
    info->dim = m->h.dim;
    info->n_cells = m->h.n_cells;
    info->n_faces = m->h.n_faces;
    info->n_boundary_faces = m->h.n_bnd;
    info->n_slots = m->h.n_slots;
    info->g_min = m->h.g_min;
    info->g_max = m->h.g_max;
    info->volume = m->h.volume;
    info->h_min = m->h.h_min;
    return DOLINC_OK;
}

dolinc_status dolinc_mesh_permutation(const dolinc_mesh *m, int64_t *new_of_old)
{
    if (!m || !new_of_old) return fail(DOLINC_ERR_INVALID_ARG, "null argument");
    std::memcpy(new_of_old, m->h.perm.data(), sizeof(int64_t) * m->h.n_cells);
    return DOLINC_OK;
}

dolinc_status dolinc_mesh_geometry(const dolinc_mesh *m, double *V, double *xc, double *S, double *w, double *d)
{
    if (!m) return fail(DOLINC_ERR_INVALID_ARG, "null mesh");
    const HostMesh &h = m->h;
    if (V) std::memcpy(V, h.V.data(), sizeof(double) * h.n_cells);
    if (xc) std::memcpy(xc, h.xc.data(), sizeof(double) * 3 * h.n_cells);
    for (int64_t i = 0; i < h.n_faces; ++i) {
        const int64_t e = h.face_ext[i];
        const double sg = h.face_flip[i] ? -1.0 : 1.0;
        for (int k = 0; k < 3; ++k) {
            if (S) S[3 * e + k] = sg * h.fS[3 * i + k];
            if (d) d[3 * e + k] = sg * h.fd[3 * i + k];
        }
        if (w) w[e] = h.face_flip[i] ? 1.0 - h.fw[i] : h.fw[i];
    }
    return DOLINC_OK;
}

dolinc_status dolinc_workspace_size(const dolinc_mesh *m, const dolinc_scheme *s, size_t *bytes)
{
    dolinc_status st = check_scheme_shape(m, s);
    if (st) return st;
    if (!bytes) return fail(DOLINC_ERR_INVALID_ARG, "null bytes");
    *bytes = ws_layout(m, s).total;
    return DOLINC_OK;
}

dolinc_status dolinc_workspace_init(void *ws, size_t bytes, dolinc_stream stream)
{
    if (!ws || bytes < 1024) return fail(DOLINC_ERR_INVALID_ARG, "workspace must hold at least 1024 bytes");
    if (((uintptr_t)ws & 255) != 0) return fail(DOLINC_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    CU(cudaMemsetAsync(ws, 0, 1024, reinterpret_cast<cudaStream_t>(stream)));
    return DOLINC_OK;
}

dolinc_status dolinc_diff_layout(const dolinc_mesh *m, const dolinc_scheme *s, int order, int64_t *offset,
                                 int *stride, int *eb, int64_t *total_bytes)
{
    dolinc_status st = check_scheme_shape(m, s);
    if (st) return st;
    if (order < 1 || order > s->n_diff) return fail(DOLINC_ERR_INVALID_ARG, "order must be in 1..n_diff");
    size_t o = 0;
    for (int mm = 1; mm <= order; ++mm) {
        const int b = elem_bytes(s->precision, mm), sd = stride_h(m->h.dim, s->nv, mm, s->precision);
        if (offset) offset[mm - 1] = (int64_t)(o / b);
        if (stride) stride[mm - 1] = sd;
        if (eb) eb[mm - 1] = b;
        o += al256((size_t)m->h.n_cells * sd * b);
    }
    if (total_bytes) *total_bytes = (int64_t)o;
    return DOLINC_OK;
}

dolinc_status dolinc_differentials(dolinc_mesh *m, const dolinc_scheme *s, const double *u, int order, void *diff,
                                   void *ws, size_t ws_bytes, dolinc_stream stream)
{
    dolinc_status st = check_scheme(m, s);
    if (st) return st;
    WsLayout L;
    if ((st = check_ws(m, s, ws, ws_bytes, L))) return st;
    if (!u || !diff) return fail(DOLINC_ERR_INVALID_ARG, "null field");
    if (order < 1 || order > s->n_diff) return fail(DOLINC_ERR_INVALID_ARG, "order must be in 1..n_diff");
    if (((uintptr_t)diff & 255) != 0) return fail(DOLINC_ERR_INVALID_ARG, "diff_dev must be 256-byte aligned");
    const PathFns *p = path_for(m, s, needed_order(*s));
    if (!p) return fail(DOLINC_ERR_UNSUPPORTED, "no kernel for this (dim, nv, order, precision)");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    timed(m, DOLINC_KERNEL_PACK, cs, [&] { p->pack(m->d, u, B(ws, L.o0[0]), nullptr, cs); });
    size_t o = 0;
    const void *prev = B(ws, L.o0[0]);
    for (int mm = 1; mm <= order; ++mm) {
        const int b = elem_bytes(s->precision, mm), sd = stride_h(m->h.dim, s->nv, mm, s->precision);
        timed(m, mm, cs, [&] {
            p->diff(m->d, mm, prev, B(diff, o), tune_for(m, s), reinterpret_cast<unsigned *>(B(ws, L.status)), cs);
            if (mm == 1) p->bnd_grad(m->d, prev, B(diff, o), cs);
        });
        prev = B(diff, o);
        o += al256((size_t)m->h.n_cells * sd * b);
    }
    return launch_check();
}

dolinc_status dolinc_reconstruct_faces(dolinc_mesh *m, const dolinc_scheme *s, const double *u, double *fL,
                                       double *fR, void *ws, size_t ws_bytes, dolinc_stream stream)
{
    dolinc_status st = check_scheme(m, s);
    if (st) return st;
    WsLayout L;
    if ((st = check_ws(m, s, ws, ws_bytes, L))) return st;
    if (!u || !fL || !fR) return fail(DOLINC_ERR_INVALID_ARG, "null field");
    const PathFns *p = path_for(m, s, needed_order(*s));
    if (!p) return fail(DOLINC_ERR_UNSUPPORTED, "no kernel for this (dim, nv, order, precision)");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    timed(m, DOLINC_KERNEL_PACK, cs, [&] { p->pack(m->d, u, B(ws, L.o0[0]), nullptr, cs); });
    run_diffs(m, p, ws, L, L.o0[0], s->n_diff, tune_for(m, s), cs);
    StageArgs a = base_args(m, s, ws, L, L.o0[0]);
    timed(m, DOLINC_KERNEL_FACES, cs, [&] { p->faces(m->d, a, fL, fR, cs); });
    return launch_check();
}

dolinc_status dolinc_residual(dolinc_mesh *m, const dolinc_scheme *s, const double *u, double *R, void *ws,
                              size_t ws_bytes, dolinc_stream stream)
{
    dolinc_status st = check_scheme(m, s);
    if (st) return st;
    WsLayout L;
    if ((st = check_ws(m, s, ws, ws_bytes, L))) return st;
    if (!u || !R) return fail(DOLINC_ERR_INVALID_ARG, "null field");
    const PathFns *p = path_for(m, s, needed_order(*s));
    if (!p) return fail(DOLINC_ERR_UNSUPPORTED, "no kernel for this (dim, nv, order, precision)");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    timed(m, DOLINC_KERNEL_PACK, cs, [&] { p->pack(m->d, u, B(ws, L.o0[0]), nullptr, cs); });
    run_diffs(m, p, ws, L, L.o0[0], s->n_diff, tune_for(m, s), cs);
    StageArgs a = base_args(m, s, ws, L, L.o0[0]);
    a.mode = 0;
    a.out = R;
    timed(m, DOLINC_KERNEL_STAGE, cs, [&] { p->stage(m->d, a, tune_for(m, s), cs); });
    return launch_check();
}

dolinc_status dolinc_rk_stage(dolinc_mesh *m, const dolinc_scheme *s, double dt, int stage, const double *u0,
                              const double *us, double *out, void *ws, size_t ws_bytes, dolinc_stream stream)
{
    static const double A[3] = {0.0, 0.75, 1.0 / 3.0}, Bc[3] = {1.0, 0.25, 2.0 / 3.0};
    dolinc_status st = check_scheme(m, s);
    if (st) return st;
    WsLayout L;
    if ((st = check_ws(m, s, ws, ws_bytes, L))) return st;
    if (!u0 || !us || !out) return fail(DOLINC_ERR_INVALID_ARG, "null field");
    if (stage < 0 || stage > 2) return fail(DOLINC_ERR_INVALID_ARG, "stage must be 0, 1 or 2");
    const PathFns *p = path_for(m, s, needed_order(*s));
    if (!p) return fail(DOLINC_ERR_UNSUPPORTED, "no kernel for this (dim, nv, order, precision)");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    timed(m, DOLINC_KERNEL_PACK, cs, [&] { p->pack(m->d, us, B(ws, L.o0[0]), nullptr, cs); });
    run_diffs(m, p, ws, L, L.o0[0], s->n_diff, tune_for(m, s), cs);
    StageArgs a = base_args(m, s, ws, L, L.o0[0]);
    a.mode = 1;
    a.u0 = u0;
    a.us = us;
    a.out = out;
    a.A = A[stage];
    a.B = Bc[stage];
    a.dt = dt;
    a.o0_next = nullptr;
    timed(m, DOLINC_KERNEL_STAGE, cs, [&] { p->stage(m->d, a, tune_for(m, s), cs); });
    return launch_check();
}

}  // extern "C"

namespace {

// One SSP-RK3 step.  The first kernel reads the step's state from u_in and, when
// u_dev differs from it, also writes it to u_dev; the stages read the step's start
// state from u_dev; the last stage writes the new state to u_out.  dolinc_rk_step
// passes one device buffer for all three.
dolinc_status rk_step_impl(dolinc_mesh *m, const dolinc_scheme *s, double dt, const double *u_in, double *u_dev,
                           double *u_out, void *ws, const WsLayout &L, cudaStream_t cs, int n_steps = 1)
{
    static const double A[3] = {0.0, 0.75, 1.0 / 3.0}, Bc[3] = {1.0, 0.25, 2.0 / 3.0};
    const PathFns *p = path_for(m, s, needed_order(*s));
    if (!p) return fail(DOLINC_ERR_UNSUPPORTED, "no kernel for this (dim, nv, order, precision)");
    double *ust = reinterpret_cast<double *>(B(ws, L.ustage));
    const Tune tn = tune_for(m, s);
    // Several steps in one call keep the state on the device: the last stage of a step
    // also writes the next step's order-0 record (the bulk-precision rounding of the new
    // FP64 state, as the pack would), so only the first step packs.
    timed(m, DOLINC_KERNEL_PACK, cs,
          [&] { p->pack(m->d, u_in, B(ws, L.o0[0]), u_dev != u_in ? u_dev : nullptr, cs); });
    bool pending = false;
    auto join = [&] {
        if (pending) cudaStreamWaitEvent(cs, m->ev_join, 0);
        pending = false;
    };
    // Paired schedule (diff lanes 2): order 1 of stage t (counted over the call's steps)
    // goes to buffer t % 2; order 2 of stage t is computed with order 1 of stage t+1 in
    // one launch, the last one after the last stage.  Returns the offset of the stage's
    // order-1 buffer.
    const bool paired = tn.diff_lpc == 2 && pair_scheme(s);
    auto o1buf = [&](int t) { return (t & 1) ? L.ord1b : L.ord[1]; };
    auto paired_diffs = [&](int t, size_t o0off) -> size_t {
        const size_t o1 = o1buf(t), o1prev = o1buf(t + 1);
        unsigned *stw = reinterpret_cast<unsigned *>(B(ws, L.status));
        const bool done = t > 0 && p->diff_pair(m->d, nullptr, nullptr, nullptr, nullptr, cs, true);
        if (done)
            timed(m, DOLINC_KERNEL_DIFF_PAIR, cs,
                  [&] { p->diff_pair(m->d, B(ws, o1prev), B(ws, L.ord[2]), B(ws, o0off), B(ws, o1), cs, false); });
        else {
            if (t > 0)
                timed(m, 2, cs, [&] { p->diff(m->d, 2, B(ws, o1prev), B(ws, L.ord[2]), tn, stw, cs); });
            timed(m, 1, cs, [&] { p->diff(m->d, 1, B(ws, o0off), B(ws, o1), tn, stw, cs); });
        }
        p->bnd_grad(m->d, B(ws, o0off), B(ws, o1), cs);
        return o1;
    };
    auto paired_tail = [&](int t_last) {   // order 2 of the last stage
        timed(m, 2, cs, [&] {
            p->diff(m->d, 2, B(ws, o1buf(t_last)), B(ws, L.ord[2]), tn, reinterpret_cast<unsigned *>(B(ws, L.status)),
                    cs);
        });
    };
    int t = 0;
    if (s->precision != DOLINC_FP64) {
        // increment form: stage k reads record o0[k], writes o0[k+1] and the accumulator
        for (int k = 0; k < n_steps; ++k) {
            const bool last = k == n_steps - 1;
            for (int sg = 0; sg < 3; ++sg, ++t) {
                join();
                size_t o1 = L.ord[1];
                if (paired) o1 = paired_diffs(t, L.o0[sg]);
                else pending = run_diffs_split(m, p, ws, L, L.o0[sg], s, tn, cs);
                StageArgs a = base_args(m, s, ws, L, L.o0[sg]);
                a.ord[1] = B(ws, o1);
                a.mode = 2;
                a.rk = sg;
                a.u0 = u_dev;
                a.out = last ? u_out : u_dev;
                a.dt = dt;
                a.dacc = reinterpret_cast<float *>(B(ws, L.dacc));
                a.rec_start = B(ws, L.o0[0]);
                a.o0_next = sg < 2 ? B(ws, L.o0[sg + 1]) : (last ? nullptr : B(ws, L.o0[0]));
                timed(m, DOLINC_KERNEL_STAGE, cs, [&] { p->stage(m->d, a, tn, cs); });
            }
        }
        join();
        if (paired) paired_tail(t - 1);
        return launch_check();
    }
    int cur = 0;
    for (int k = 0; k < n_steps; ++k) {
        const bool last = k == n_steps - 1;
        for (int sg = 0; sg < 3; ++sg, ++t) {
            join();
            size_t o1 = L.ord[1];
            if (paired) o1 = paired_diffs(t, L.o0[cur]);
            else pending = run_diffs_split(m, p, ws, L, L.o0[cur], s, tn, cs);
            StageArgs a = base_args(m, s, ws, L, L.o0[cur]);
            a.ord[1] = B(ws, o1);
            a.mode = 1;
            a.u0 = u_dev;
            a.us = sg == 0 ? u_dev : ust;
            a.out = sg < 2 ? ust : (last ? u_out : u_dev);
            a.A = A[sg];
            a.B = Bc[sg];
            a.dt = dt;
            a.o0_next = (sg == 2 && last) ? nullptr : B(ws, L.o0[1 - cur]);
            timed(m, DOLINC_KERNEL_STAGE, cs, [&] { p->stage(m->d, a, tn, cs); });
            cur = 1 - cur;
        }
    }
    join();
    if (paired) paired_tail(t - 1);
    return launch_check();
}

}  // namespace

extern "C" {

dolinc_status dolinc_rk_step(dolinc_mesh *m, const dolinc_scheme *s, double dt, double *u, void *ws,
                             size_t ws_bytes, dolinc_stream stream)
{
    dolinc_status st = check_scheme(m, s);
    if (st) return st;
    WsLayout L;
    if ((st = check_ws(m, s, ws, ws_bytes, L))) return st;
    if (!u) return fail(DOLINC_ERR_INVALID_ARG, "null field");
    return rk_step_impl(m, s, dt, u, u, u, ws, L, reinterpret_cast<cudaStream_t>(stream));
}

dolinc_status dolinc_rk_steps(dolinc_mesh *m, const dolinc_scheme *s, double dt, int n_steps, double *u, void *ws,
                              size_t ws_bytes, dolinc_stream stream)
{
    dolinc_status st = check_scheme(m, s);
    if (st) return st;
    WsLayout L;
    if ((st = check_ws(m, s, ws, ws_bytes, L))) return st;
    if (!u) return fail(DOLINC_ERR_INVALID_ARG, "null field");
    if (n_steps < 1) return fail(DOLINC_ERR_INVALID_ARG, "n_steps must be at least 1");
    return rk_step_impl(m, s, dt, u, u, u, ws, L, reinterpret_cast<cudaStream_t>(stream), n_steps);
}

dolinc_status dolinc_rk_step_host(dolinc_mesh *m, const dolinc_scheme *s, double dt, double *u_host, double *u_dev,
                                  void *ws, size_t ws_bytes, dolinc_stream stream)
{
    dolinc_status st = check_scheme(m, s);
    if (st) return st;
    WsLayout L;
    if ((st = check_ws(m, s, ws, ws_bytes, L))) return st;
    if (!u_host || !u_dev) return fail(DOLINC_ERR_INVALID_ARG, "null field");
    if (u_host == u_dev) return fail(DOLINC_ERR_INVALID_ARG, "u_host and u_dev must be different buffers");
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, u_dev) != cudaSuccess ||
        (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged)) {
        cudaGetLastError();
        return fail(DOLINC_ERR_INVALID_ARG, "u_dev must be device memory");
    }
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    // page-locked, mapped host memory: the kernels read and write it in place
    void *mapped = nullptr;
    if (cudaHostGetDevicePointer(&mapped, u_host, 0) == cudaSuccess && mapped) {
        double *uh = static_cast<double *>(mapped);
        return rk_step_impl(m, s, dt, uh, u_dev, uh, ws, L, cs);
    }
    cudaGetLastError();
    // other host memory: copied in and out on the stream
    const size_t bytes = (size_t)m->h.n_cells * s->nv * sizeof(double);
    CU(cudaMemcpyAsync(u_dev, u_host, bytes, cudaMemcpyHostToDevice, cs));
    if ((st = rk_step_impl(m, s, dt, u_dev, u_dev, u_dev, ws, L, cs))) return st;
    CU(cudaMemcpyAsync(u_host, u_dev, bytes, cudaMemcpyDeviceToHost, cs));
    return DOLINC_OK;
}

dolinc_status dolinc_profile_enable(dolinc_mesh *m, int enable)
{
    if (!m) return fail(DOLINC_ERR_INVALID_ARG, "null mesh");
    for (auto &r : m->recs) m->pool.push_back(r.a), m->pool.push_back(r.b);
    m->recs.clear();
    for (int k = 0; k < DOLINC_KERNEL_COUNT; ++k) m->prof_ms[k] = 0, m->prof_n[k] = 0;
    m->prof = enable != 0;
    return DOLINC_OK;
}

dolinc_status dolinc_profile_read(dolinc_mesh *m, double *ms, int64_t *launches)
{
    if (!m) return fail(DOLINC_ERR_INVALID_ARG, "null mesh");
    for (auto &r : m->recs) {
        CU(cudaEventSynchronize(r.b));
        float t = 0;
        CU(cudaEventElapsedTime(&t, r.a, r.b));
        m->prof_ms[r.kind] += t;
        m->prof_n[r.kind] += 1;
        m->pool.push_back(r.a);
        m->pool.push_back(r.b);
    }
    m->recs.clear();
    for (int k = 0; k < DOLINC_KERNEL_COUNT; ++k) {
        if (ms) ms[k] = m->prof_ms[k];
        if (launches) launches[k] = m->prof_n[k];
    }
    return DOLINC_OK;
}

dolinc_status dolinc_autotune(dolinc_mesh *m, const dolinc_scheme *s, const double *u, void *ws, size_t ws_bytes,
                              const char *cache_path, dolinc_stream stream, dolinc_tuning *out)
{
    dolinc_status st = check_scheme(m, s);
    if (st) return st;
    WsLayout L;
    if ((st = check_ws(m, s, ws, ws_bytes, L))) return st;
    if (!u) return fail(DOLINC_ERR_INVALID_ARG, "null field");
    const PathFns *p = path_for(m, s, needed_order(*s));
    if (!p) return fail(DOLINC_ERR_UNSUPPORTED, "no kernel for this (dim, nv, order, precision)");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    cudaDeviceProp prop;
    CU(cudaGetDeviceProperties(&prop, m->device));
    const std::string key = std::string(prop.name) + "|" + scheme_key(m, s);
    Tune best;
    bool cached = false;
    if (cache_path) {
        std::ifstream in(cache_path);
        std::string line;
        while (std::getline(in, line)) {
            std::istringstream ls(line);
            std::string k;
            Tune t;
            if (std::getline(ls, k, '\t') && (ls >> t.diff_lpc >> t.diff_block >> t.stage_lpc >> t.stage_block) &&
                k == key) {
                best = t;
                cached = true;
            }
        }
    }
    double best_diff = 0, best_stage = 0;
    if (!cached) {
        const bool prof = m->prof;
        m->prof = false;
        p->pack(m->d, u, B(ws, L.o0[0]), nullptr, cs);
        cudaEvent_t e0, e1;
        CU(cudaEventCreate(&e0));
        CU(cudaEventCreate(&e1));
        auto time_it = [&](auto &&launch) {
            for (int i = 0; i < 2; ++i) launch();
            cudaEventRecord(e0, cs);
            for (int i = 0; i < 5; ++i) launch();
            cudaEventRecord(e1, cs);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            return ms / 5.0;
        };
        // diff shapes: lanes 1/4/8, tiled (0), persistent pipelined (-1/-4 with 128/256
        // threads); stage shapes: lanes 1/4/8, tiled, persistent pipelined (-1 with tiles
        // of 64/128 cells)
        const int lpcs[7] = {1, 4, 8, 0, -1, -4, -2}, blocks[3] = {64, 128, 256};
        double bd = 1e30, bs = 1e30;
        for (int li = 0; li < 7; ++li)
            for (int bi = 0; bi < 3; ++bi) {
                Tune t;
                t.diff_lpc = t.stage_lpc = lpcs[li];
                t.diff_block = t.stage_block = blocks[bi];
                const bool diff_ok = (lpcs[li] >= 0 || blocks[bi] >= 128) && lpcs[li] != -2;
                const bool stage_ok = lpcs[li] == -2 || (lpcs[li] >= -1 && (lpcs[li] >= 0 || blocks[bi] <= 128));
                if (!diff_ok) t.diff_lpc = best.diff_lpc, t.diff_block = best.diff_block;
                if (diff_ok) {
                    double td = time_it([&] {
                        for (int mm = 1; mm <= s->n_diff; ++mm)
                            p->diff(m->d, mm, B(ws, mm == 1 ? L.o0[0] : L.ord[mm - 1]), B(ws, L.ord[mm]), t,
                                    reinterpret_cast<unsigned *>(B(ws, L.status)), cs);
                    });
                    if (td < bd) bd = td, best.diff_lpc = t.diff_lpc, best.diff_block = t.diff_block;
                }
                if (!stage_ok) continue;
                // the stage as rk_step runs it (middle stage), on scratch outputs
                StageArgs a = base_args(m, s, ws, L, L.o0[0]);
                double *scratch = reinterpret_cast<double *>(B(ws, L.ustage));
                a.u0 = a.us = a.out = scratch;
                a.dt = 0.0;
                if (s->precision != DOLINC_FP64) {
                    a.mode = 2;
                    a.rk = 1;
                    a.dacc = reinterpret_cast<float *>(B(ws, L.dacc));
                    a.rec_start = B(ws, L.o0[0]);
                    a.o0_next = B(ws, L.o0[2]);
                } else {
                    a.mode = 1;
                    a.A = 0.75;
                    a.B = 0.25;
                    a.o0_next = B(ws, L.o0[1]);
                }
                double tsg = time_it([&] { p->stage(m->d, a, t, cs); });
                if (tsg < bs) bs = tsg, best.stage_lpc = t.stage_lpc, best.stage_block = t.stage_block;
            }
        // the paired schedule (lanes 2): a stage's passes are one paired launch (order 2
        // of the previous stage with its own order 1), against lanes 1's two passes
        if (pair_scheme(s) && best.diff_lpc == 1) {
            bool launched = true;
            launched = p->diff_pair(m->d, nullptr, nullptr, nullptr, nullptr, cs, true);
            const double tp = launched ? time_it([&] {
                p->diff_pair(m->d, B(ws, L.ord[1]), B(ws, L.ord[2]), B(ws, L.o0[0]), B(ws, L.ord1b), cs, false);
            }) : 1e30;
            if (launched && tp < bd) bd = tp, best.diff_lpc = 2;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        m->prof = prof;
        best_diff = bd;
        best_stage = bs;
        CU(cudaMemsetAsync(B(ws, L.status), 0, 1024, cs));   // the timing runs may have flagged garbage
        CU(cudaStreamSynchronize(cs));
        if (cache_path) {
            std::ofstream o(cache_path, std::ios::app);
            o << key << '\t' << best.diff_lpc << ' ' << best.diff_block << ' ' << best.stage_lpc << ' '
              << best.stage_block << '\n';
        }
    }
    m->tuned[scheme_key(m, s)] = best;
    if (out) {
        out->diff_lanes = best.diff_lpc;
        out->diff_block = best.diff_block;
        out->stage_lanes = best.stage_lpc;
        out->stage_block = best.stage_block;
        out->from_cache = cached ? 1 : 0;
        out->diff_ms = best_diff;
        out->stage_ms = best_stage;
    }
    return launch_check();
}

// ------------------------------------------------------------------ indicator and network
namespace {
dolinc_status indicator_prep(dolinc_mesh *m, const dolinc_scheme *s, const double *u, void *ws, size_t ws_bytes,
                             cudaStream_t cs, WsLayout &L, const IndicatorFns **fi)
{
    dolinc_status st = check_scheme(m, s);
    if (st) return st;
    if ((st = check_ws(m, s, ws, ws_bytes, L))) return st;
    if (!u) return fail(DOLINC_ERR_INVALID_ARG, "null field");
    if (s->flux != DOLINC_FLUX_RUSANOV || s->n_diff < 2)
        return fail(DOLINC_ERR_INVALID_ARG, "the indicator needs an Euler scheme with n_diff >= 2");
    const PathFns *p = path_for(m, s, needed_order(*s));
    if (!p) return fail(DOLINC_ERR_UNSUPPORTED, "no kernel for this (dim, nv, order, precision)");
    const int nsr = needed_order(*s) > 2 ? needed_order(*s) : 2;
    *fi = &g_ind[indicator_index(m->h.dim, nsr, s->precision)];
    if (!(*fi)->criterion) return fail(DOLINC_ERR_UNSUPPORTED, "no indicator kernel for this scheme");
    timed(m, DOLINC_KERNEL_PACK, cs, [&] { p->pack(m->d, u, B(ws, L.o0[0]), nullptr, cs); });
    run_diffs(m, p, ws, L, L.o0[0], s->n_diff, tune_for(m, s), cs);
    return DOLINC_OK;
}

uint64_t splitmix(uint64_t &x)
{
    uint64_t z = (x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

dolinc_status mlp_scratch(dolinc_mlp *m, long long n)
{
    if (n <= m->cap) return DOLINC_OK;
    m->free_scratch();
    const size_t h = sizeof(float) * (size_t)n * MLP_H;
    CU(cudaMalloc(&m->A1, h));
    CU(cudaMalloc(&m->A2, h));
    CU(cudaMalloc(&m->A3, h));
    CU(cudaMalloc(&m->z, sizeof(float) * (size_t)n));
    CU(cudaMalloc(&m->dZa, h));
    CU(cudaMalloc(&m->dZb, h));
    m->cap = n;
    return DOLINC_OK;
}

// loss and gradient of one batch into m->g (and *loss_dev); forward on the bf16 weights
dolinc_status mlp_grad(dolinc_mlp *m, const float *x, const uint8_t *y, long long n, float pw, float *loss_dev,
                       cudaStream_t cs)
{
    dolinc_status st = mlp_scratch(m, n);
    if (st) return st;
    const float *q = m->q;
    launch_quantize(m->theta, m->q, cs);
    launch_dense_fwd(x, MLP_IN, q + OFF_W1, q + OFF_B1, MLP_H, n, m->A1, true, cs);
    launch_dense_fwd(m->A1, MLP_H, q + OFF_W2, q + OFF_B2, MLP_H, n, m->A2, true, cs);
    launch_dense_fwd(m->A2, MLP_H, q + OFF_W3, q + OFF_B3, MLP_H, n, m->A3, true, cs);
    launch_dense_fwd(m->A3, MLP_H, q + OFF_W4, q + OFF_B4, 1, n, m->z, false, cs);
    CU(cudaMemsetAsync(m->g, 0, sizeof(float) * MLP_PARAMS, cs));
    if (loss_dev) CU(cudaMemsetAsync(loss_dev, 0, sizeof(float), cs));
    float *dz = m->dZa;
    launch_bce(m->z, y, n, pw, dz, loss_dev, cs);
    launch_dense_bwd_w(dz, m->A3, MLP_H, 1, n, m->g + OFF_W4, m->g + OFF_B4, cs);
    launch_dense_bwd_x(dz, q + OFF_W4, MLP_H, 1, n, m->A3, m->dZb, cs);              // dZ3
    launch_dense_bwd_w(m->dZb, m->A2, MLP_H, MLP_H, n, m->g + OFF_W3, m->g + OFF_B3, cs);
    launch_dense_bwd_x(m->dZb, q + OFF_W3, MLP_H, MLP_H, n, m->A2, m->dZa, cs);     // dZ2
    launch_dense_bwd_w(m->dZa, m->A1, MLP_H, MLP_H, n, m->g + OFF_W2, m->g + OFF_B2, cs);
    launch_dense_bwd_x(m->dZa, q + OFF_W2, MLP_H, MLP_H, n, m->A1, m->dZb, cs);     // dZ1
    launch_dense_bwd_w(m->dZb, x, MLP_IN, MLP_H, n, m->g + OFF_W1, m->g + OFF_B1, cs);
    return launch_check();
}
}  // namespace

dolinc_status dolinc_criterion(dolinc_mesh *m, const dolinc_scheme *s, const double *u, uint8_t *flags, double kappa,
                               double eps, void *ws, size_t ws_bytes, dolinc_stream stream)
{
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    WsLayout L;
    const IndicatorFns *fi = nullptr;
    if (!flags) return fail(DOLINC_ERR_INVALID_ARG, "null flags");
    dolinc_status st = indicator_prep(m, s, u, ws, ws_bytes, cs, L, &fi);
    if (st) return st;
    StageArgs a = base_args(m, s, ws, L, L.o0[0]);
    fi->criterion(m->d, a, kappa, eps, flags, cs);
    return launch_check();
}

dolinc_status dolinc_indicator_features(dolinc_mesh *m, const dolinc_scheme *s, const double *u, float *x24,
                                        void *ws, size_t ws_bytes, dolinc_stream stream)
{
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    WsLayout L;
    const IndicatorFns *fi = nullptr;
    if (!x24) return fail(DOLINC_ERR_INVALID_ARG, "null feature buffer");
    dolinc_status st = indicator_prep(m, s, u, ws, ws_bytes, cs, L, &fi);
    if (st) return st;
    StageArgs a = base_args(m, s, ws, L, L.o0[0]);
    float *own = reinterpret_cast<float *>(B(ws, L.ustage));   // 6 floats per cell fit in nv doubles
    fi->own_features(m->d, a, own, cs);
    launch_gather24(m->d, own, x24, cs);
    return launch_check();
}

dolinc_status dolinc_mlp_create(dolinc_mlp **out, uint64_t seed)
{
    if (!out) return fail(DOLINC_ERR_INVALID_ARG, "null output handle");
    *out = nullptr;
    dolinc_mlp *m = new (std::nothrow) dolinc_mlp();
    if (!m) return fail(DOLINC_ERR_OOM, "host allocation");
    cudaGetDevice(&m->device);
    std::vector<float> th(MLP_PARAMS, 0.0f);
    uint64_t st = seed;
    const int sizes[4][3] = {{OFF_W1, MLP_H, MLP_IN}, {OFF_W2, MLP_H, MLP_H}, {OFF_W3, MLP_H, MLP_H}, {OFF_W4, 1, MLP_H}};
    for (auto &L : sizes) {
        const float lim = std::sqrt(6.0f / (float)L[2]);              // He-uniform
        for (int i = 0; i < L[1] * L[2]; ++i) {
            double u01 = (double)(splitmix(st) >> 11) * (1.0 / 9007199254740992.0);
            th[L[0] + i] = (float)((2.0 * u01 - 1.0) * lim);
        }
    }
    auto al = [&](void **p, size_t b) { return cudaMalloc(p, b); };
    cudaError_t e = cudaSuccess;
    for (float **p : {&m->theta, &m->q, &m->m, &m->v, &m->g})
        if (e == cudaSuccess) e = al((void **)p, sizeof(float) * MLP_PARAMS);
    if (e == cudaSuccess) e = al((void **)&m->loss, sizeof(float));
    if (e == cudaSuccess) e = al((void **)&m->frag, sizeof(uint2) * N_FRAGS * 32);
    if (e == cudaSuccess) e = cudaMemcpy(m->theta, th.data(), sizeof(float) * MLP_PARAMS, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->m, 0, sizeof(float) * MLP_PARAMS);
    if (e == cudaSuccess) e = cudaMemset(m->v, 0, sizeof(float) * MLP_PARAMS);
    if (e != cudaSuccess) {
        delete m;
        return fail(e == cudaErrorMemoryAllocation ? DOLINC_ERR_OOM : DOLINC_ERR_CUDA,
                    std::string("dolinc_mlp_create: ") + cudaGetErrorString(e));
    }
    *out = m;
    return DOLINC_OK;
}

void dolinc_mlp_destroy(dolinc_mlp *m) { delete m; }

dolinc_status dolinc_mlp_get_params(const dolinc_mlp *m, float *host)
{
    if (!m || !host) return fail(DOLINC_ERR_INVALID_ARG, "null argument");
    CU(cudaMemcpy(host, m->theta, sizeof(float) * MLP_PARAMS, cudaMemcpyDeviceToHost));
    return DOLINC_OK;
}

dolinc_status dolinc_mlp_set_params(dolinc_mlp *m, const float *host)
{
    if (!m || !host) return fail(DOLINC_ERR_INVALID_ARG, "null argument");
    CU(cudaMemcpy(m->theta, host, sizeof(float) * MLP_PARAMS, cudaMemcpyHostToDevice));
    m->frag_ok = false;
    return DOLINC_OK;
}

dolinc_status dolinc_mlp_forward(dolinc_mlp *m, const float *x, int64_t n, float *logits, uint8_t *flags,
                                 dolinc_stream stream)
{
    if (!m || !x || n < 0 || (!logits && !flags)) return fail(DOLINC_ERR_INVALID_ARG, "bad argument");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    if (!m->frag_ok) {
        launch_mlp_frags(m->theta, m->frag, cs);
        m->frag_ok = true;
    }
    if (n > 0) launch_mlp_infer(m->frag, m->theta, x, n, logits, flags, cs);
    return launch_check();
}

dolinc_status dolinc_mlp_loss_grad(dolinc_mlp *m, const float *x, const uint8_t *y, int64_t n, float pos_weight,
                                   float *grad, float *loss, dolinc_stream stream)
{
    if (!m || !x || !y || n <= 0) return fail(DOLINC_ERR_INVALID_ARG, "bad argument");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    dolinc_status st = mlp_grad(m, x, y, n, pos_weight, loss, cs);
    if (st) return st;
    if (grad) CU(cudaMemcpyAsync(grad, m->g, sizeof(float) * MLP_PARAMS, cudaMemcpyDeviceToDevice, cs));
    return DOLINC_OK;
}

dolinc_status dolinc_mlp_train_step(dolinc_mlp *m, const float *x, const uint8_t *y, int64_t n, float lr,
                                    float pos_weight, float *loss, dolinc_stream stream)
{
    if (!m || !x || !y || n <= 0) return fail(DOLINC_ERR_INVALID_ARG, "bad argument");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    dolinc_status st = mlp_grad(m, x, y, n, pos_weight, loss, cs);
    if (st) return st;
    m->step += 1;
    launch_adam(m->theta, m->m, m->v, m->g, MLP_PARAMS, lr, m->step, cs);
    m->frag_ok = false;
    return launch_check();
}

dolinc_status dolinc_indicator_infer(dolinc_mesh *me, const dolinc_scheme *s, dolinc_mlp *net, const double *u,
                                     float *x24, uint8_t *flags, float *logits, void *ws, size_t ws_bytes,
                                     dolinc_stream stream)
{
    if (x24) {
        dolinc_status st = dolinc_indicator_features(me, s, u, x24, ws, ws_bytes, stream);
        if (st) return st;
        return dolinc_mlp_forward(net, x24, me->h.n_cells, logits, flags, stream);
    }
    // without an input buffer: the network gathers its inputs itself (no round trip)
    if (!net || (!logits && !flags)) return fail(DOLINC_ERR_INVALID_ARG, "bad argument");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    WsLayout L;
    const IndicatorFns *fi = nullptr;
    dolinc_status st = indicator_prep(me, s, u, ws, ws_bytes, cs, L, &fi);
    if (st) return st;
    StageArgs a = base_args(me, s, ws, L, L.o0[0]);
    float *own = reinterpret_cast<float *>(B(ws, L.ustage));
    fi->own_features(me->d, a, own, cs);
    if (!net->frag_ok) {
        launch_mlp_frags(net->theta, net->frag, cs);
        net->frag_ok = true;
    }
    launch_mlp_infer_fused(net->frag, net->theta, me->d, own, logits, flags, cs);
    return launch_check();
}

// ------------------------------------------------------------------ batches
dolinc_status dolinc_batch_create(dolinc_mesh *const *meshes, int n, dolinc_batch **out)
{
    for (int b = 0; meshes && b < n; ++b)
        if (meshes[b] && !meshes[b]->h.minv.empty())
            return fail(DOLINC_ERR_UNSUPPORTED, "batches take no mesh with the skewness correction on");
    if (!out) return fail(DOLINC_ERR_INVALID_ARG, "null output handle");
    *out = nullptr;
    if (!meshes || n <= 0) return fail(DOLINC_ERR_INVALID_ARG, "empty batch");
    for (int b = 0; b < n; ++b) {
        if (!meshes[b]) return fail(DOLINC_ERR_INVALID_ARG, "null mesh in batch");
        if (meshes[b]->h.dim != meshes[0]->h.dim) return fail(DOLINC_ERR_INVALID_ARG, "meshes of different dimension");
        if (meshes[b]->d.n_bv > 0)
            return fail(DOLINC_ERR_UNSUPPORTED, "batched steps take no Dirichlet/Neumann boundary faces");
    }
    dolinc_batch *bt = new (std::nothrow) dolinc_batch();
    if (!bt) return fail(DOLINC_ERR_OOM, "host allocation");
    bt->arena = new (std::nothrow) dolinc_mesh();
    if (!bt->arena) {
        delete bt;
        return fail(DOLINC_ERR_OOM, "host allocation");
    }
    HostMesh &H = bt->arena->h;
    H.dim = meshes[0]->h.dim;
    H.off.push_back(0);
    H.g_min = 1e300;
    H.g_max = 0;
    H.h_min = 1e300;
    std::vector<int32_t> cell_mesh;
    bt->n = n;
    bt->cell_off.push_back(0);
    try {
        for (int b = 0; b < n; ++b) {
            const HostMesh &h = meshes[b]->h;
            const int64_t co = H.n_cells, so = H.n_slots, fo = H.n_faces;
            if (co + h.n_cells > ((int64_t)1 << 30) || fo + h.n_faces > ((int64_t)1 << 29)) {
                delete bt;
                return fail(DOLINC_ERR_INVALID_ARG, "batch too large (2^30 cells / 2^29 faces)");
            }
            for (int64_t p : h.perm) H.perm.push_back(p + co);
            H.V.insert(H.V.end(), h.V.begin(), h.V.end());
            H.xc.insert(H.xc.end(), h.xc.begin(), h.xc.end());
            H.cw.insert(H.cw.end(), h.cw.begin(), h.cw.end());
            for (int64_t c = 0; c < h.n_cells; ++c) H.off.push_back((int32_t)(h.off[c + 1] + so));
            for (int32_t v : h.snb) H.snb.push_back((int32_t)(v + co));
            for (uint32_t w : h.sword) H.sword.push_back(slot_word((int64_t)(w >> 2) + fo, (w & 2) != 0, (int)(w & 1)));
            H.ss.insert(H.ss.end(), h.ss.begin(), h.ss.end());
            for (int64_t v : h.fo) H.fo.push_back(v + co);
            for (int64_t v : h.fn) H.fn.push_back(v < 0 ? -1 : v + co);
            for (int64_t v : h.face_ext) H.face_ext.push_back(v + fo);
            H.face_flip.insert(H.face_flip.end(), h.face_flip.begin(), h.face_flip.end());
            H.fS.insert(H.fS.end(), h.fS.begin(), h.fS.end());
            H.fxf.insert(H.fxf.end(), h.fxf.begin(), h.fxf.end());
            H.fd.insert(H.fd.end(), h.fd.begin(), h.fd.end());
            H.fw.insert(H.fw.end(), h.fw.begin(), h.fw.end());
            H.fg.insert(H.fg.end(), h.fg.begin(), h.fg.end());
            H.n_cells += h.n_cells;
            H.n_faces += h.n_faces;
            H.n_slots += h.n_slots;
            H.n_bnd += h.n_bnd;
            H.volume += h.volume;
            H.g_min = std::min(H.g_min, h.g_min);
            H.g_max = std::max(H.g_max, h.g_max);
            H.h_min = std::min(H.h_min, h.h_min);
            cell_mesh.insert(cell_mesh.end(), (size_t)h.n_cells, (int32_t)b);
            bt->cell_off.push_back(H.n_cells);
        }
    } catch (const std::bad_alloc &) {
        delete bt;
        return fail(DOLINC_ERR_OOM, "host allocation while concatenating the batch");
    }
    dolinc_status st = upload_mesh(bt->arena);
    if (!st) st = upload(bt->arena, cell_mesh, &bt->cell_mesh);
    if (st) {
        delete bt;
        return st;
    }
    *out = bt;
    return DOLINC_OK;
}

void dolinc_batch_destroy(dolinc_batch *b) { delete b; }

dolinc_status dolinc_batch_set_spin_limit(dolinc_batch *b, unsigned polls)
{
    if (!b) return fail(DOLINC_ERR_INVALID_ARG, "null batch");
    b->spin_limit = polls;
    return DOLINC_OK;
}

dolinc_status dolinc_batch_info(const dolinc_batch *b, int64_t *n_cells, int64_t *cell_offsets)
{
    if (!b) return fail(DOLINC_ERR_INVALID_ARG, "null batch");
    if (n_cells) *n_cells = b->arena->h.n_cells;
    if (cell_offsets) std::memcpy(cell_offsets, b->cell_off.data(), sizeof(int64_t) * (b->n + 1));
    return DOLINC_OK;
}

dolinc_status dolinc_batch_workspace_size(const dolinc_batch *b, const dolinc_scheme *s, size_t *bytes)
{
    if (!b) return fail(DOLINC_ERR_INVALID_ARG, "null batch");
    return dolinc_workspace_size(b->arena, s, bytes);
}

namespace {
dolinc_status batch_launch_step(dolinc_batch *bt, const dolinc_scheme *s, const BatchFns *bf, const double *dt,
                                double *u, void *ws, const WsLayout &L, cudaStream_t cs)
{
    static const double A[3] = {0.0, 0.75, 1.0 / 3.0}, Bc[3] = {1.0, 0.25, 2.0 / 3.0};
    dolinc_mesh *m = bt->arena;
    double *ust = reinterpret_cast<double *>(B(ws, L.ustage));
    int cur = 0;
    for (int sg = 0; sg < 3; ++sg) {
        StageArgs a = base_args(m, s, ws, L, L.o0[cur]);
        a.mode = 1;
        a.u0 = u;
        a.us = sg == 0 ? u : ust;
        a.out = sg == 2 ? u : ust;
        a.A = A[sg];
        a.B = Bc[sg];
        a.o0_next = sg == 2 ? nullptr : B(ws, L.o0[1 - cur]);
        BatchArgs b{};
        b.pack_src = sg == 0 ? u : nullptr;
        b.ord[0] = B(ws, L.o0[cur]);
        for (int mm = 1; mm <= MAXN; ++mm) b.ord[mm] = B(ws, L.ord[mm]);
        b.n_diff = s->n_diff;
        b.cell_mesh = bt->cell_mesh;
        b.dt_tab = dt;
        b.bar = reinterpret_cast<unsigned *>(B(ws, L.status + 256));
        b.spin_limit = bt->spin_limit;
        cudaError_t e = bf->launch(m->d, a, b, bt->grid, bt->block, cs);
        if (e != cudaSuccess) return fail(DOLINC_ERR_CUDA, std::string("cooperative launch: ") + cudaGetErrorString(e));
        cur = 1 - cur;
    }
    return DOLINC_OK;
}

dolinc_status batch_prepare(dolinc_batch *bt, const dolinc_scheme *s, const double *dt, double *u, void *ws,
                            size_t ws_bytes, WsLayout &L, const BatchFns **bf)
{
    dolinc_mesh *m = bt->arena;
    dolinc_status st = check_scheme(m, s);
    if (st) return st;
    if ((st = check_ws(m, s, ws, ws_bytes, L))) return st;
    if (!u || !dt) return fail(DOLINC_ERR_INVALID_ARG, "null field or time steps");
    if (s->limiter != DOLINC_LIMIT_NONE) return fail(DOLINC_ERR_UNSUPPORTED, "batched steps take no limiter");
    const int ns = needed_order(*s);
    if (ns > 2) return fail(DOLINC_ERR_UNSUPPORTED, "batched steps support stencils of DOLINC order <= 2");
    std::call_once(g_once, init_paths);
    *bf = &g_batch[batch_index(m->h.dim, s->nv, ns, s->precision)];
    if (!(*bf)->launch) return fail(DOLINC_ERR_UNSUPPORTED, "no batched kernel for this scheme");
    if (bt->grid <= 0) {
        int sms = 0;
        CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device));
        const int per = (*bf)->blocks_per_sm(bt->block);
        if (per <= 0) return fail(DOLINC_ERR_UNSUPPORTED, "batched kernel does not fit on an SM");
        bt->grid = per * sms;
    }
    return DOLINC_OK;
}
}  // namespace

dolinc_status dolinc_batch_rk_step(dolinc_batch *bt, const dolinc_scheme *s, const double *dt, double *u, void *ws,
                                   size_t ws_bytes, int use_graph, dolinc_stream stream)
{
    if (!bt) return fail(DOLINC_ERR_INVALID_ARG, "null batch");
    WsLayout L;
    const BatchFns *bf = nullptr;
    dolinc_status st = batch_prepare(bt, s, dt, u, ws, ws_bytes, L, &bf);
    if (st) return st;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    if (!use_graph) return batch_launch_step(bt, s, bf, dt, u, ws, L, cs);
    std::ostringstream k;
    k << (const void *)u << '|' << ws << '|' << (const void *)dt << '|' << scheme_key(bt->arena, s) << '|' << s->k << ','
      << s->r << ',' << s->flux << ',' << s->gamma << ',' << s->adv[0] << ',' << s->adv[1] << ',' << s->adv[2] << '|'
      << bt->block << ',' << bt->grid << ',' << bt->spin_limit;
    if (!bt->exec || bt->gkey != k.str()) {
        if (bt->exec) {
            cudaGraphExecDestroy(bt->exec);
            bt->exec = nullptr;
        }
        // capture on a private stream (the caller's may be the legacy stream, which
        // cannot be captured); the graph is then launched on the caller's stream
        if (!bt->cap) CU(cudaStreamCreateWithFlags(&bt->cap, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        CU(cudaStreamBeginCapture(bt->cap, cudaStreamCaptureModeThreadLocal));
        dolinc_status ls = batch_launch_step(bt, s, bf, dt, u, ws, L, bt->cap);
        cudaError_t e = cudaStreamEndCapture(bt->cap, &g);
        cudaGetLastError();
        if (ls) {
            if (g) cudaGraphDestroy(g);
            return ls;
        }
        if (e != cudaSuccess) return fail(DOLINC_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&bt->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            bt->exec = nullptr;
            return fail(DOLINC_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        }
        bt->gkey = k.str();
    }
    CU(cudaGraphLaunch(bt->exec, cs));
    return DOLINC_OK;
}

dolinc_status dolinc_batch_autotune(dolinc_batch *bt, const dolinc_scheme *s, const double *dt, double *u, void *ws,
                                    size_t ws_bytes, dolinc_stream stream, int *block_out, int *grid_out,
                                    double *ms_out)
{
    if (!bt) return fail(DOLINC_ERR_INVALID_ARG, "null batch");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    const int blocks[3] = {64, 128, 256};
    const double fracs[2] = {1.0, 0.5};
    int best_b = 256, best_g = 0;
    double best = 1e30;
    int sms = 0;
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, bt->arena->device));
    // time on a copy of the state so the caller's field is left as it was
    const size_t ubytes = sizeof(double) * (size_t)s->nv * (size_t)bt->arena->h.n_cells;
    WsLayout L0 = ws_layout(bt->arena, s);
    if (!ws || ws_bytes < L0.total) return fail(DOLINC_ERR_INVALID_ARG, "workspace too small");
    std::vector<char> keep(ubytes);
    CU(cudaMemcpyAsync(keep.data(), u, ubytes, cudaMemcpyDeviceToHost, cs));
    CU(cudaStreamSynchronize(cs));
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    for (int bi = 0; bi < 3; ++bi)
        for (int fi = 0; fi < 2; ++fi) {
            bt->block = blocks[bi];
            bt->grid = 0;
            WsLayout L;
            const BatchFns *bf = nullptr;
            dolinc_status st = batch_prepare(bt, s, dt, u, ws, ws_bytes, L, &bf);
            if (st) continue;
            bt->grid = std::max(1, (int)(bt->grid * fracs[fi]));
            if (batch_launch_step(bt, s, bf, dt, u, ws, L, cs)) continue;
            cudaEventRecord(e0, cs);
            for (int r = 0; r < 3; ++r) batch_launch_step(bt, s, bf, dt, u, ws, L, cs);
            cudaEventRecord(e1, cs);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms / 3 < best) best = ms / 3, best_b = bt->block, best_g = bt->grid;
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    bt->block = best_b;
    bt->grid = best_g;
    CU(cudaMemcpyAsync(u, keep.data(), ubytes, cudaMemcpyHostToDevice, cs));
    CU(cudaMemsetAsync(ws, 0, 1024, cs));
    CU(cudaStreamSynchronize(cs));
    if (block_out) *block_out = best_b;
    if (grid_out) *grid_out = best_g;
    if (ms_out) *ms_out = best;
    return launch_check();
}

dolinc_status dolinc_set_tuning(dolinc_mesh *m, const dolinc_scheme *s, const dolinc_tuning *t)
{
    dolinc_status st = check_scheme_shape(m, s);
    if (st) return st;
    if (!t) return fail(DOLINC_ERR_INVALID_ARG, "null tuning");
    auto ok = [](int l, int b) {
        if (l == 0) return b == 64 || b == 128 || b == 256;
        return (l == 1 || l == 4 || l == 8) && b >= 32 && b <= 256 && b % 32 == 0;
    };
    const bool diff_pipe = ((t->diff_lanes == -1 || t->diff_lanes == -4) && (t->diff_block == 128 || t->diff_block == 256)) ||
                           (t->diff_lanes == 2 && t->diff_block >= 32 && t->diff_block <= 256 && t->diff_block % 32 == 0);
    const bool stage_pipe = (t->stage_lanes == -1 && (t->stage_block == 64 || t->stage_block == 128)) ||
                            (t->stage_lanes == -2 && (t->stage_block == 64 || t->stage_block == 128 || t->stage_block == 256));
    if (!(ok(t->diff_lanes, t->diff_block) || diff_pipe) || !(ok(t->stage_lanes, t->stage_block) || stage_pipe))
        return fail(DOLINC_ERR_INVALID_ARG,
                    "lanes 1, 4 or 8 with blocks a multiple of 32 in 32..256, or lanes 0 (tiled) with 64/128/256; "
                    "differential passes also lanes -1 / -4 (persistent pipelined) with 128/256 or lanes 2 (paired "
                    "schedule) with blocks as lanes 1, the stage "
                    "lanes -1 (persistent pipelined) with tiles of 64/128 cells or -2 (face-centric) with 64/128/256");
    Tune x;
    x.diff_lpc = t->diff_lanes;
    x.diff_block = t->diff_block;
    x.stage_lpc = t->stage_lanes;
    x.stage_block = t->stage_block;
    m->tuned[scheme_key(m, s)] = x;
    return DOLINC_OK;
}

dolinc_status dolinc_set_boundary_values(dolinc_mesh *m, int nv, const double *values)
{
    if (!m) return fail(DOLINC_ERR_INVALID_ARG, "null mesh");
    if (nv < 1 || nv > 5) return fail(DOLINC_ERR_INVALID_ARG, "nv must be in 1..5");
    if (m->d.n_bv == 0) return fail(DOLINC_ERR_INVALID_ARG, "the mesh has no Dirichlet/Neumann faces");
    if (!values) return fail(DOLINC_ERR_INVALID_ARG, "null values");
    const HostMesh &h = m->h;
    const int nb = m->d.n_bv;
    std::vector<double> v64((size_t)nv * nb);
    std::vector<float> v32((size_t)nv * nb);
    for (int64_t f = 0; f < h.n_faces; ++f) {
        if (h.fkind[f] < 2) continue;
        const int b = m->bidx_h[f];
        const int64_t ext = h.face_ext[f];
        for (int v = 0; v < nv; ++v) {
            double x = values[(int64_t)v * h.n_faces + ext];
            // a Neumann gradient is given along the caller's outward normal, which is
            // the internal one (a boundary face's owner is its only cell)
            if (!std::isfinite(x)) return fail(DOLINC_ERR_INVALID_ARG, "non-finite boundary value");
            v64[(size_t)v * nb + b] = x;
            v32[(size_t)v * nb + b] = (float)x;
        }
    }
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != m->device) CU(cudaSetDevice(m->device));
    dolinc_status st = DOLINC_OK;
    const double *p64 = nullptr;
    const float *p32 = nullptr;
    if (!(st = upload(m, v64, &p64))) st = upload(m, v32, &p32);
    if (cur != m->device) cudaSetDevice(cur);
    if (st) return st;
    m->d.bval64 = p64;
    m->d.bval32 = p32;
    m->bv_nv = nv;
    return DOLINC_OK;
}

dolinc_status dolinc_set_flags(dolinc_mesh *m, const uint8_t *flags)
{
    if (!m) return fail(DOLINC_ERR_INVALID_ARG, "null mesh");
    m->flags = flags;
    return DOLINC_OK;
}

dolinc_status dolinc_sync_status(dolinc_mesh *m, void *ws, dolinc_stream stream)
{
    if (!m || !ws) return fail(DOLINC_ERR_INVALID_ARG, "null argument");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    unsigned h = 0;
    CU(cudaMemcpyAsync(&h, ws, sizeof h, cudaMemcpyDeviceToHost, cs));
    CU(cudaStreamSynchronize(cs));
    CU(cudaMemsetAsync(ws, 0, 1024, cs));      // status and the batch barrier words
    CU(cudaStreamSynchronize(cs));
    if (h & 2u) return fail(DOLINC_ERR_DEVICE_TIMEOUT, "a device-side wait gave up");
    if (h & 1u) return fail(DOLINC_ERR_NONFINITE, "a stage produced NaN or Inf");
    return DOLINC_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ partitioned meshes
namespace {

// Record rows of `n` cells: gather (dst row i = src row idx[i]) or scatter (dst row
// idx[i] = src row i), moved in words of wbytes (a divisor of the record size; rows
// and buffers start at multiples of it).
__global__ void __launch_bounds__(256) k_halo_copy(const unsigned char *__restrict__ src, unsigned char *__restrict__ dst,
                                                   const int32_t *__restrict__ idx, long long n, int words,
                                                   int wbytes, int gather)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * words) return;
    const long long i = t / words;
    const int w = (int)(t % words);
    const long long a = gather ? (long long)idx[i] : i, b = gather ? i : (long long)idx[i];
    const size_t rb = (size_t)words * wbytes;
    const unsigned char *ps = src + a * rb;
    unsigned char *pd = dst + b * rb;
    switch (wbytes) {
    case 16: reinterpret_cast<uint4 *>(pd)[w] = reinterpret_cast<const uint4 *>(ps)[w]; break;
    case 8: reinterpret_cast<uint2 *>(pd)[w] = reinterpret_cast<const uint2 *>(ps)[w]; break;
    case 4: reinterpret_cast<unsigned *>(pd)[w] = reinterpret_cast<const unsigned *>(ps)[w]; break;
    case 2: reinterpret_cast<unsigned short *>(pd)[w] = reinterpret_cast<const unsigned short *>(ps)[w]; break;
    default: pd[w] = ps[w]; break;
    }
}

size_t rec_bytes(const dolinc_mesh *m, const dolinc_scheme *s, int order)
{
    return (size_t)stride_h(m->h.dim, s->nv, order, s->precision) * elem_bytes(s->precision, order);
}

void halo_copy(const void *src, void *dst, const int32_t *idx, size_t n, size_t rb, bool gather, cudaStream_t cs)
{
    if (n == 0) return;
    int wb = 16;
    while (rb % wb) wb /= 2;
    const int words = (int)(rb / wb);
    const long long tot = (long long)n * words;
    k_halo_copy<<<(int)((tot + 255) / 256), 256, 0, cs>>>(static_cast<const unsigned char *>(src),
                                                          static_cast<unsigned char *>(dst), idx, (long long)n,
                                                          words, wb, gather ? 1 : 0);
}

// Offset of the record buffer of `order` that the current stage reads.
size_t part_rec_off(const dolinc_mesh *m, const dolinc_scheme *s, const WsLayout &L, int order)
{
    const PartState &P = *m->part;
    if (order > 0) return L.ord[order];
    return s->precision != DOLINC_FP64 ? L.o0[P.stage] : L.o0[P.cur];
}

// Packs the own cells' records of `order` for the peers and describes the exchange.
void part_request(dolinc_mesh *m, const dolinc_scheme *s, void *ws, const WsLayout &L, int order, cudaStream_t cs,
                  dolinc_halo *h)
{
    PartState &P = *m->part;
    const size_t rb = rec_bytes(m, s, order);
    halo_copy(B(ws, part_rec_off(m, s, L, order)), B(ws, L.hsend), P.send_dev, P.plan.send_cells.size(), rb, true,
              cs);
    P.order = order;
    h->pending = 1;
    h->order = order;
    h->record_bytes = rb;
    h->send_dev = B(ws, L.hsend);
    h->recv_dev = B(ws, L.hrecv);
}

// Highest order exchanged per stage: each pass's input, and every order the stage reads.
int part_top_order(const dolinc_scheme *s)
{
    const int need = needed_order(*s);
    return std::max(s->n_diff - 1, need);
}

// Runs the step from just after the exchange of P.order to the next exchange point
// (or the end of the step).
dolinc_status part_advance(dolinc_mesh *m, const dolinc_scheme *s, void *ws, const WsLayout &L, cudaStream_t cs,
                           dolinc_halo *h)
{
    static const double A[3] = {0.0, 0.75, 1.0 / 3.0}, Bc[3] = {1.0, 0.25, 2.0 / 3.0};
    PartState &P = *m->part;
    const PathFns *p = path_for(m, s, needed_order(*s));
    if (!p) return fail(DOLINC_ERR_UNSUPPORTED, "no kernel for this (dim, nv, order, precision)");
    const Tune tn = tune_for(m, s);
    const int top = part_top_order(s);
    const size_t o0off = part_rec_off(m, s, L, 0);
    for (int mm = P.order + 1; mm <= s->n_diff; ++mm) {
        timed(m, mm, cs, [&] {
            p->diff(m->d, mm, B(ws, mm == 1 ? o0off : L.ord[mm - 1]), B(ws, L.ord[mm]), tn,
                    reinterpret_cast<unsigned *>(B(ws, L.status)), cs);
            if (mm == 1) p->bnd_grad(m->d, B(ws, o0off), B(ws, L.ord[1]), cs);
        });
        if (mm <= top) {
            part_request(m, s, ws, L, mm, cs, h);
            return launch_check();
        }
    }
    // every order the stage reads is in place on the ghosts: the stage kernel
    const int sg = P.stage;
    StageArgs a = base_args(m, s, ws, L, o0off);
    a.dt = P.dt;
    a.u0 = P.u;
    if (s->precision != DOLINC_FP64) {
        a.mode = 2;
        a.rk = sg;
        a.out = P.u;
        a.dacc = reinterpret_cast<float *>(B(ws, L.dacc));
        a.rec_start = B(ws, L.o0[0]);
        a.o0_next = sg == 2 ? nullptr : B(ws, L.o0[sg + 1]);
    } else {
        double *ust = reinterpret_cast<double *>(B(ws, L.ustage));
        a.mode = 1;
        a.us = sg == 0 ? P.u : ust;
        a.out = sg == 2 ? P.u : ust;
        a.A = A[sg];
        a.B = Bc[sg];
        a.o0_next = sg == 2 ? nullptr : B(ws, L.o0[1 - P.cur]);
    }
    timed(m, DOLINC_KERNEL_STAGE, cs, [&] { p->stage(m->d, a, tn, cs); });
    if (sg < 2) {
        P.stage = sg + 1;
        P.cur = 1 - P.cur;
        part_request(m, s, ws, L, 0, cs, h);
        return launch_check();
    }
    P.active = false;
    P.order = -1;
    h->pending = 0;
    h->order = -1;
    h->record_bytes = 0;
    h->send_dev = h->recv_dev = nullptr;
    return launch_check();
}

dolinc_status plan_from_desc(const dolinc_mesh_desc *desc, const int32_t *part_of_cell, int n_parts, int part,
                             HostMesh &g, PartPlan &plan)
{
    if (!desc || !part_of_cell) return fail(DOLINC_ERR_INVALID_ARG, "null descriptor or part_of_cell");
    std::string err;
    try {
        err = build_host_mesh(*desc, g);
    } catch (const std::bad_alloc &) {
        return fail(DOLINC_ERR_OOM, "host allocation while building the mesh");
    }
    if (!err.empty()) return fail(DOLINC_ERR_MESH, err);
    std::vector<int32_t> part_lib(g.n_cells);
    for (int64_t c = 0; c < g.n_cells; ++c) part_lib[g.perm[c]] = part_of_cell[c];
    err = plan_part(g, part_lib, n_parts, part, plan);
    if (!err.empty()) return fail(DOLINC_ERR_INVALID_ARG, err);
    return DOLINC_OK;
}

void fill_sizes(const PartPlan &p, dolinc_part_sizes *z)
{
    z->n_local = (int64_t)p.cells.size();
    z->n_owned = 0;
    for (uint8_t o : p.owned) z->n_owned += o;
    z->n_faces = (int64_t)p.faces.size();
    z->n_peers = (int32_t)p.peers.size();
    z->n_send = (int64_t)p.send_cells.size();
    z->n_recv = (int64_t)p.recv_cells.size();
}

}  // namespace

extern "C" {

dolinc_status dolinc_partition(const dolinc_mesh_desc *desc, int n_parts, int32_t *part_of_cell)
{
    if (!desc || !part_of_cell) return fail(DOLINC_ERR_INVALID_ARG, "null argument");
    if (n_parts < 1 || n_parts > desc->n_cells) return fail(DOLINC_ERR_INVALID_ARG, "n_parts must be in 1..n_cells");
    dolinc_mesh_desc d = *desc;
    d.renumber = DOLINC_RENUMBER_MORTON;
    HostMesh g;
    std::string err;
    try {
        err = build_host_mesh(d, g);
    } catch (const std::bad_alloc &) {
        return fail(DOLINC_ERR_OOM, "host allocation while building the mesh");
    }
    if (!err.empty()) return fail(DOLINC_ERR_MESH, err);
    for (int64_t c = 0; c < g.n_cells; ++c) part_of_cell[c] = (int32_t)((g.perm[c] * (int64_t)n_parts) / g.n_cells);
    return DOLINC_OK;
}

dolinc_status dolinc_part_plan(const dolinc_mesh_desc *desc, const int32_t *part_of_cell, int n_parts, int part,
                               dolinc_part_sizes *sizes, int64_t *local_cells, uint8_t *owned, int32_t *peers,
                               int64_t *send_off, int64_t *send_cells, int64_t *recv_off, int64_t *recv_cells)
{
    if (!sizes) return fail(DOLINC_ERR_INVALID_ARG, "null sizes");
    HostMesh g;
    PartPlan p;
    dolinc_status st = plan_from_desc(desc, part_of_cell, n_parts, part, g, p);
    if (st) return st;
    fill_sizes(p, sizes);
    if (local_cells) {
        std::vector<int64_t> old_of_new(g.n_cells);
        for (int64_t c = 0; c < g.n_cells; ++c) old_of_new[g.perm[c]] = c;
        for (size_t j = 0; j < p.cells.size(); ++j) local_cells[j] = old_of_new[p.cells[j]];
    }
    if (owned) std::memcpy(owned, p.owned.data(), p.owned.size());
    if (peers) std::memcpy(peers, p.peers.data(), sizeof(int32_t) * p.peers.size());
    if (send_off) std::memcpy(send_off, p.send_off.data(), sizeof(int64_t) * p.send_off.size());
    if (recv_off) std::memcpy(recv_off, p.recv_off.data(), sizeof(int64_t) * p.recv_off.size());
    if (send_cells) std::memcpy(send_cells, p.send_cells.data(), sizeof(int64_t) * p.send_cells.size());
    if (recv_cells) std::memcpy(recv_cells, p.recv_cells.data(), sizeof(int64_t) * p.recv_cells.size());
    return DOLINC_OK;
}

dolinc_status dolinc_mesh_create_part(const dolinc_mesh_desc *desc, const int32_t *part_of_cell, int n_parts,
                                      int part, dolinc_mesh **out)
{
    if (!out) return fail(DOLINC_ERR_INVALID_ARG, "null output handle");
    *out = nullptr;
    HostMesh g;
    auto ps = std::unique_ptr<PartState>(new (std::nothrow) PartState());
    if (!ps) return fail(DOLINC_ERR_OOM, "host allocation");
    dolinc_status st = plan_from_desc(desc, part_of_cell, n_parts, part, g, ps->plan);
    if (st) return st;
    dolinc_mesh *m = new (std::nothrow) dolinc_mesh();
    if (!m) return fail(DOLINC_ERR_OOM, "host allocation");
    try {
        slice_host_mesh(g, ps->plan, m->h);
    } catch (const std::bad_alloc &) {
        delete m;
        return fail(DOLINC_ERR_OOM, "host allocation while slicing the part");
    }
    if ((st = upload_mesh(m))) {
        delete m;
        return st;
    }
    std::vector<int32_t> sc(ps->plan.send_cells.begin(), ps->plan.send_cells.end());
    std::vector<int32_t> rc(ps->plan.recv_cells.begin(), ps->plan.recv_cells.end());
    sc.push_back(0);                            // never empty
    rc.push_back(0);
    if ((st = upload(m, sc, &ps->send_dev)) || (st = upload(m, rc, &ps->recv_dev))) {
        delete m;
        return st;
    }
    m->part = std::move(ps);
    *out = m;
    return DOLINC_OK;
}

dolinc_status dolinc_mesh_part_sizes(const dolinc_mesh *m, dolinc_part_sizes *sizes)
{
    if (!m || !sizes) return fail(DOLINC_ERR_INVALID_ARG, "null argument");
    if (!m->part) return fail(DOLINC_ERR_INVALID_ARG, "not a part mesh");
    fill_sizes(m->part->plan, sizes);
    return DOLINC_OK;
}

dolinc_status dolinc_part_step_begin(dolinc_mesh *m, const dolinc_scheme *s, double dt, double *u, void *ws,
                                     size_t ws_bytes, dolinc_stream stream, dolinc_halo *h)
{
    dolinc_status st = check_scheme(m, s);
    if (st) return st;
    if (!m->part) return fail(DOLINC_ERR_INVALID_ARG, "not a part mesh (dolinc_mesh_create_part)");
    if (!h || !u) return fail(DOLINC_ERR_INVALID_ARG, "null field or halo");
    WsLayout L;
    if ((st = check_ws(m, s, ws, ws_bytes, L))) return st;
    const PathFns *p = path_for(m, s, needed_order(*s));
    if (!p) return fail(DOLINC_ERR_UNSUPPORTED, "no kernel for this (dim, nv, order, precision)");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    PartState &P = *m->part;
    P.active = true;
    P.stage = 0;
    P.cur = 0;
    P.dt = dt;
    P.u = u;
    timed(m, DOLINC_KERNEL_PACK, cs, [&] { p->pack(m->d, u, B(ws, L.o0[0]), nullptr, cs); });
    part_request(m, s, ws, L, 0, cs, h);
    return launch_check();
}

dolinc_status dolinc_part_step_continue(dolinc_mesh *m, const dolinc_scheme *s, void *ws, size_t ws_bytes,
                                        dolinc_stream stream, dolinc_halo *h)
{
    dolinc_status st = check_scheme(m, s);
    if (st) return st;
    if (!m->part || !m->part->active) return fail(DOLINC_ERR_INVALID_ARG, "no partitioned step in progress");
    if (!h) return fail(DOLINC_ERR_INVALID_ARG, "null halo");
    WsLayout L;
    if ((st = check_ws(m, s, ws, ws_bytes, L))) return st;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    PartState &P = *m->part;
    halo_copy(B(ws, L.hrecv), B(ws, part_rec_off(m, s, L, P.order)), P.recv_dev, P.plan.recv_cells.size(),
              rec_bytes(m, s, P.order), false, cs);
    return part_advance(m, s, ws, L, cs, h);
}

}  // extern "C"

extern "C" {

dolinc_status dolinc_mesh_set_skew_correction(dolinc_mesh *m, int enable)
{
    if (!m) return fail(DOLINC_ERR_INVALID_ARG, "null mesh");
    if (enable && m->d.n_bv > 0)
        return fail(DOLINC_ERR_UNSUPPORTED, "the skewness correction takes no Dirichlet/Neumann faces");
    std::vector<uint8_t> ghost;
    if (m->part) {
        ghost.resize(m->h.n_cells);
        for (size_t j = 0; j < ghost.size(); ++j) ghost[j] = m->part->plan.owned[j] ? 0 : 1;
    }
    std::string err;
    try {
        err = apply_skew(m->h, enable != 0, m->part ? &ghost : nullptr);
    } catch (const std::bad_alloc &) {
        return fail(DOLINC_ERR_OOM, "host allocation");
    }
    if (!err.empty()) {
        apply_skew(m->h, false, nullptr);
        return fail(DOLINC_ERR_MESH, err);
    }
    std::vector<double> sk64, ck64;
    std::vector<float> sk32, ck32;
    weight_tables(m->h, sk64, sk32, ck64, ck32);
    int cur = 0;
    cudaGetDevice(&cur);
    CU(cudaSetDevice(m->device));
    CU(cudaDeviceSynchronize());
    auto put = [&](const void *dst, const void *src, size_t bytes) {
        return cudaMemcpy(const_cast<void *>(dst), src, bytes, cudaMemcpyHostToDevice);
    };
    CU(put(m->d.slotk64, sk64.data(), sizeof(double) * sk64.size()));
    CU(put(m->d.slotk32, sk32.data(), sizeof(float) * sk32.size()));
    CU(put(m->d.cellk64, ck64.data(), sizeof(double) * ck64.size()));
    CU(put(m->d.cellk32, ck32.data(), sizeof(float) * ck32.size()));
    if (enable) {
        const int64_t nf = m->h.n_faces;
        std::vector<double> d64(4 * nf, 0.0);
        std::vector<float> d32(4 * nf, 0.0f);
        for (int64_t f = 0; f < nf; ++f)
            for (int k = 0; k < 3; ++k) {
                d64[4 * f + k] = m->h.sdelta[3 * f + k];
                d32[4 * f + k] = (float)m->h.sdelta[3 * f + k];
            }
        dolinc_status st;
        if ((st = upload(m, d64, &m->d.fdelta64)) || (st = upload(m, d32, &m->d.fdelta32))) {
            cudaSetDevice(cur);
            return st;
        }
    } else {
        m->d.fdelta64 = nullptr;
        m->d.fdelta32 = nullptr;
    }
    CU(cudaSetDevice(cur));
    return DOLINC_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ semi-implicit step
struct dolinc_implicit {
    dolinc_mesh *m = nullptr;
    dolinc_scheme s{};
    double dt = 0.0, theta = 1.0;
    double rel_tol = 1e-10;
    int max_iter = 1000;
    unsigned spin_limit = 1u << 23;
    int warm = 0;                        // initial guess of a step's first solve: 0, 1 previous, 2 extrapolated
    int grid = 0, device = 0;
    int ell = 0;                         // ELL width of the rows (0: per slot)
    int64_t n = 0, ns = 0, ne = 0;       // cells, slots, row entries
    int sms = 0;
    void *mem = nullptr;
    void *rows = nullptr;                // nbr and off (their own allocation: the layout can change)
    int32_t *nbr = nullptr;
    double *off = nullptr, *diag = nullptr, *bscale = nullptr;
    double *vec[7] = {};                 // x r rh p v s t
    double *R = nullptr, *Rn = nullptr, *un = nullptr;
    double *xw[3] = {};                  // the steps' first solutions, rotated between steps
    int xw_last = 0, xw_have = 0;        // buffer of the last step's solution; solutions kept (0..2)
    double *part = nullptr;
    double *scal = nullptr;              // ctrl block: scalars (256 B), then barrier words and status (512 B)
    double *life = nullptr;              // [2] iterations and solves since creation (not reset per step)
    unsigned *bar = nullptr;
    cudaStream_t last = nullptr;
    ~dolinc_implicit()
    {
        if (!mem && !rows) return;
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(device);
        if (mem) cudaFree(mem);
        if (rows) cudaFree(rows);
        cudaSetDevice(cur);
    }
};

namespace {
constexpr size_t kImpCtrl = 768;     // scalars 256 B + barrier words [0], [32], [64] and status [96]
constexpr int kImpMaxBlocksPerSm = 8;

// (Re)builds the rows in layout ell (ELL width, 0 = per slot) and sizes the grid for it:
// waits for the device, frees the old rows, assembles, waits again.
dolinc_status imp_build_rows(dolinc_implicit *imp, int ell)
{
    const dolinc_mesh *m = imp->m;
    CU(cudaDeviceSynchronize());
    if (imp->rows) {
        cudaFree(imp->rows);
        imp->rows = nullptr;
    }
    imp->ell = ell;
    imp->ne = ell ? (int64_t)ell * imp->n : imp->ns;
    const size_t e4 = (4 * (size_t)std::max<int64_t>(imp->ne, 1) + 255) / 256 * 256;
    cudaError_t e = cudaMalloc(&imp->rows, e4 + 8 * (size_t)std::max<int64_t>(imp->ne, 1));
    if (e != cudaSuccess) {
        cudaGetLastError();
        imp->rows = nullptr;
        return fail(DOLINC_ERR_OOM, std::string("implicit solver rows: ") + cudaGetErrorString(e));
    }
    imp->nbr = static_cast<int32_t *>(imp->rows);
    imp->off = reinterpret_cast<double *>(static_cast<char *>(imp->rows) + e4);
    const int64_t need = (imp->n + IMP_BLOCK - 1) / IMP_BLOCK;
    const int bps = std::min(std::max(imp_solve_blocks_per_sm(ell), 1), kImpMaxBlocksPerSm);
    imp->grid = (int)std::max<int64_t>(1, std::min(need, (int64_t)imp->sms * bps));
    const dolinc_scheme *s = &imp->s;
    launch_imp_assemble(m->d, needed_order(*s), s->k, s->r, s->adv[0], s->adv[1], s->adv[2], imp->dt, imp->theta, ell,
                        imp->nbr, imp->off, imp->diag, imp->bscale, nullptr);
    dolinc_status st = launch_check();
    if (st) return st;
    CU(cudaDeviceSynchronize());
    return DOLINC_OK;
}
}

extern "C" {

dolinc_status dolinc_implicit_create(dolinc_mesh *m, const dolinc_scheme *s, double dt, double theta,
                                     dolinc_implicit **out)
{
    if (!out) return fail(DOLINC_ERR_INVALID_ARG, "null output");
    *out = nullptr;
    dolinc_status st = check_scheme(m, s);
    if (st) return st;
    if (s->flux != DOLINC_FLUX_UPWIND || s->nv != 1)
        return fail(DOLINC_ERR_UNSUPPORTED, "the semi-implicit step is for linear advection (UPWIND flux, nv = 1)");
    if (m->d.n_bv > 0)
        return fail(DOLINC_ERR_UNSUPPORTED, "the semi-implicit step takes zero-gradient boundary faces only");
    if (m->part) return fail(DOLINC_ERR_UNSUPPORTED, "the semi-implicit step solves over a whole mesh, not a part");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(DOLINC_ERR_INVALID_ARG, "dt must be positive and finite");
    if (!(theta >= 0.0 && theta <= 1.0)) return fail(DOLINC_ERR_INVALID_ARG, "theta must be in [0, 1]");
    std::unique_ptr<dolinc_implicit> imp(new dolinc_implicit);
    imp->m = m;
    imp->s = *s;
    imp->dt = dt;
    imp->theta = theta;
    imp->device = m->device;
    imp->n = m->h.n_cells;
    imp->ns = m->h.n_slots;
    int cur = 0;
    CU(cudaGetDevice(&cur));
    CU(cudaSetDevice(m->device));
    CU(cudaDeviceGetAttribute(&imp->sms, cudaDevAttrMultiProcessorCount, m->device));
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t n8 = al(8 * (size_t)std::max<int64_t>(imp->n, 1));
    const size_t pb = al(8 * IMP_NRED * (size_t)imp->sms * kImpMaxBlocksPerSm);
    const size_t total = 15 * n8 + pb + kImpCtrl + 256;    // 7 vectors, diag, bscale, R, Rn, un, 3 kept solutions
    cudaError_t e = cudaMalloc(&imp->mem, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaSetDevice(cur);
        return fail(DOLINC_ERR_OOM, std::string("implicit solver memory: ") + cudaGetErrorString(e));
    }
    char *q = static_cast<char *>(imp->mem);
    auto take = [&](size_t b) { char *r = q; q += b; return r; };
    imp->diag = reinterpret_cast<double *>(take(n8));
    imp->bscale = reinterpret_cast<double *>(take(n8));
    for (auto &v : imp->vec) v = reinterpret_cast<double *>(take(n8));
    imp->R = reinterpret_cast<double *>(take(n8));
    imp->Rn = reinterpret_cast<double *>(take(n8));
    imp->un = reinterpret_cast<double *>(take(n8));
    for (auto &w : imp->xw) w = reinterpret_cast<double *>(take(n8));
    imp->part = reinterpret_cast<double *>(take(pb));
    imp->scal = reinterpret_cast<double *>(take(kImpCtrl));
    imp->bar = reinterpret_cast<unsigned *>(reinterpret_cast<char *>(imp->scal) + 256);
    imp->life = reinterpret_cast<double *>(take(256));
    CU(cudaMemset(imp->mem, 0, total));
    if ((st = imp_build_rows(imp.get(), 0))) {       // per-slot rows (measured faster than ELL)
        cudaSetDevice(cur);
        return st;
    }
    CU(cudaSetDevice(cur));
    *out = imp.release();
    return DOLINC_OK;
}

dolinc_status dolinc_implicit_set_layout(dolinc_implicit *imp, int ell)
{
    if (!imp) return fail(DOLINC_ERR_INVALID_ARG, "null solver");
    if (!(ell == 0 || ((ell == 4 || ell == 6 || ell == 8) && ell >= imp->m->d.max_slots)))
        return fail(DOLINC_ERR_INVALID_ARG, "layout must be 0 (per slot) or an ELL width 4, 6 or 8 covering every cell");
    int cur = 0;
    CU(cudaGetDevice(&cur));
    CU(cudaSetDevice(imp->device));
    dolinc_status st = imp_build_rows(imp, ell);
    CU(cudaSetDevice(cur));
    return st;
}

int dolinc_implicit_layout(const dolinc_implicit *imp) { return imp ? imp->ell : -1; }

void dolinc_implicit_destroy(dolinc_implicit *imp) { delete imp; }

dolinc_status dolinc_implicit_set_solver(dolinc_implicit *imp, double rel_tol, int max_iter, unsigned spin_limit,
                                         int warm_start)
{
    if (!imp) return fail(DOLINC_ERR_INVALID_ARG, "null solver");
    if (!(rel_tol >= 0.0) || !std::isfinite(rel_tol)) return fail(DOLINC_ERR_INVALID_ARG, "rel_tol must be >= 0");
    if (max_iter < 1) return fail(DOLINC_ERR_INVALID_ARG, "max_iter must be >= 1");
    if (warm_start < 0 || warm_start > 2) return fail(DOLINC_ERR_INVALID_ARG, "warm_start must be 0, 1 or 2");
    int cur = 0;
    CU(cudaGetDevice(&cur));
    CU(cudaSetDevice(imp->device));
    CU(cudaDeviceSynchronize());
    imp->xw_have = 0;                                   // the next warm start begins from 0
    CU(cudaSetDevice(cur));
    imp->rel_tol = rel_tol;
    imp->max_iter = max_iter;
    imp->spin_limit = spin_limit;
    imp->warm = warm_start;
    return DOLINC_OK;
}

dolinc_status dolinc_implicit_step(dolinc_implicit *imp, double *u, int n_outer, void *ws, size_t ws_bytes,
                                   dolinc_stream stream)
{
    if (!imp || !u) return fail(DOLINC_ERR_INVALID_ARG, "null solver or field");
    if (n_outer < 1) return fail(DOLINC_ERR_INVALID_ARG, "n_outer must be >= 1");
    if (!imp->rows) return fail(DOLINC_ERR_INVALID_ARG, "the solver has no rows (a failed dolinc_implicit_set_layout)");
    dolinc_mesh *m = imp->m;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    CU(cudaMemsetAsync(imp->scal, 0, kImpCtrl, cs));
    if (n_outer > 1) CU(cudaMemcpyAsync(imp->un, u, 8 * (size_t)imp->n, cudaMemcpyDeviceToDevice, cs));
    ImpSolve a{};
    a.n = (int)imp->n;
    a.row = m->d.off;
    a.nbr = imp->nbr;
    a.off = imp->off;
    a.bscale = imp->bscale;
    a.inv_dt = 1.0 / imp->dt;
    a.theta = imp->theta;
    a.u = u;
    a.x = imp->vec[0];
    a.r = imp->vec[1];
    a.rh = imp->vec[2];
    a.p = imp->vec[3];
    a.v = imp->vec[4];
    a.s = imp->vec[5];
    a.t = imp->vec[6];
    a.part = imp->part;
    a.scal = imp->scal;
    a.life = imp->life;
    a.bar = imp->bar;
    a.status = imp->bar + 96;
    a.tol2 = imp->rel_tol * imp->rel_tol;
    a.max_iter = imp->max_iter;
    a.spin_limit = imp->spin_limit;
    for (int k = 0; k < n_outer; ++k) {
        double *Rk = k == 0 ? imp->Rn : imp->R;
        dolinc_status st = dolinc_residual(m, &imp->s, u, Rk, ws, ws_bytes, stream);
        if (st) return st;
        a.R = Rk;
        a.Rn = k == 0 ? nullptr : imp->Rn;
        a.un = k == 0 ? nullptr : imp->un;
        // warm start of the step's first solve from the last steps' first solutions (the
        // solution goes to the third buffer, which then becomes the last); the
        // outer corrections start from 0
        const bool first = imp->warm && k == 0;
        a.warm = first ? std::min(imp->warm, imp->xw_have) : 0;
        a.x1 = imp->xw[imp->xw_last];
        a.x2 = imp->xw[(imp->xw_last + 2) % 3];
        a.x = first ? imp->xw[(imp->xw_last + 1) % 3] : imp->vec[0];
        cudaError_t e = cudaSuccess;
        timed(m, DOLINC_KERNEL_SOLVE, cs, [&] { e = launch_imp_solve(a, imp->ell, imp->grid, cs); });
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(DOLINC_ERR_CUDA, std::string("cooperative launch: ") + cudaGetErrorString(e));
        }
        if (first) {
            imp->xw_last = (imp->xw_last + 1) % 3;
            imp->xw_have = std::min(imp->xw_have + 1, 2);
        }
    }
    imp->last = cs;
    return launch_check();
}

dolinc_status dolinc_implicit_info(dolinc_implicit *imp, dolinc_solve_info *info)
{
    if (!imp || !info) return fail(DOLINC_ERR_INVALID_ARG, "null argument");
    double sc[SC_COUNT], life[2];
    unsigned status = 0;
    CU(cudaStreamSynchronize(imp->last));
    CU(cudaMemcpy(sc, imp->scal, sizeof sc, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(life, imp->life, sizeof life, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(&status, imp->bar + 96, sizeof status, cudaMemcpyDeviceToHost));
    info->iterations = (int)sc[SC_ITERS];
    info->solves = (int)sc[SC_SOLVES];
    info->breakdown = (status & 4u) ? 1 : 0;
    info->converged = (status & (2u | 4u | 8u)) ? 0 : 1;
    info->rel_residual = sc[SC_BB] > 0.0 ? std::sqrt(sc[SC_RR] / sc[SC_BB]) : 0.0;
    info->total_iterations = (int64_t)life[0];
    info->total_solves = (int64_t)life[1];
    if (status & 2u) return fail(DOLINC_ERR_DEVICE_TIMEOUT, "a device-side wait gave up");
    return DOLINC_OK;
}

dolinc_status dolinc_implicit_rows(const dolinc_implicit *imp, int32_t *row_offsets, int32_t *nbr, double *off,
                                   double *diag)
{
    if (!imp || !row_offsets || !nbr || !off || !diag) return fail(DOLINC_ERR_INVALID_ARG, "null argument");
    if (!imp->rows) return fail(DOLINC_ERR_INVALID_ARG, "the solver has no rows (a failed dolinc_implicit_set_layout)");
    const dolinc_mesh *m = imp->m;
    CU(cudaDeviceSynchronize());
    std::memcpy(row_offsets, m->h.off.data(), sizeof(int32_t) * (size_t)(imp->n + 1));
    std::vector<int32_t> nb(imp->ne);
    std::vector<double> of(imp->ne);
    CU(cudaMemcpy(nb.data(), imp->nbr, 4 * (size_t)imp->ne, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(of.data(), imp->off, 8 * (size_t)imp->ne, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(diag, imp->diag, 8 * (size_t)imp->n, cudaMemcpyDeviceToHost));
    for (int64_t c = 0; c < imp->n; ++c)
        for (int32_t k = row_offsets[c]; k < row_offsets[c + 1]; ++k) {
            const int64_t e = imp->ell ? (int64_t)(k - row_offsets[c]) * imp->n + c : k;
            nbr[k] = nb[e];
            off[k] = of[e] * diag[c];
        }
    return DOLINC_OK;
}

}  // extern "C"
