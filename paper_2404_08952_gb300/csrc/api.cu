// C ABI of the DOLINC stage library (include/dolinc.h).
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <chrono>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/dolinc.h"
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

#define CU(call)                                                                                          \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess)                                                                            \
            return fail(e_ == cudaErrorMemoryAllocation ? DOLINC_ERR_OOM : DOLINC_ERR_CUDA,               \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                              \
    } while (0)

PathFns g_paths[N_PATHS];
std::once_flag g_once;

void init_paths()
{
    std::memset(g_paths, 0, sizeof g_paths);
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

struct dolinc_mesh {
    HostMesh h;
    DevMesh d{};
    int device = 0;
    std::vector<void *> allocs;
    const uint8_t *flags = nullptr;
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
    ~dolinc_mesh()
    {
        for (auto &r : recs) pool.push_back(r.a), pool.push_back(r.b);
        for (auto e : pool) cudaEventDestroy(e);
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(device);
        for (void *p : allocs) cudaFree(p);
        cudaSetDevice(cur);
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
    if (s.limiter != DOLINC_LIMIT_NONE && need < 2) need = 2;
    return need < 1 ? 1 : need;
}

dolinc_status check_scheme(const dolinc_mesh *m, const dolinc_scheme *s)
{
    if (!m || !s) return fail(DOLINC_ERR_INVALID_ARG, "null mesh or scheme");
    if (s->k < 1 || s->r < 0 || s->r >= s->k) return fail(DOLINC_ERR_INVALID_ARG, "bad stencil (k, r)");
    if (s->n_diff < 1 || s->n_diff > MAXN) return fail(DOLINC_ERR_INVALID_ARG, "n_diff must be in 1..4");
    if (needed_order(*s) > s->n_diff)
        return fail(DOLINC_ERR_INVALID_ARG, "stencil (k, r) / limiter needs more differential orders than n_diff");
    if (s->precision < DOLINC_FP64 || s->precision > DOLINC_FP32_BF16)
        return fail(DOLINC_ERR_INVALID_ARG, "unknown precision");
    if (s->limiter < DOLINC_LIMIT_NONE || s->limiter > DOLINC_LIMIT_ENO3_FLAGGED)
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
    if (s->limiter == DOLINC_LIMIT_ENO3_FLAGGED && !m->flags)
        return fail(DOLINC_ERR_INVALID_ARG, "flagged limiter without flags (dolinc_set_flags)");
    return DOLINC_OK;
}

int elem_bytes(int prec, int m) { return prec == DOLINC_FP64 ? 8 : (prec == DOLINC_FP32_BF16 && m >= 2 ? 2 : 4); }
int ncoef_h(int dim, int m) { return dim == 2 ? m + 1 : (m + 1) * (m + 2) / 2; }
int stride_h(int dim, int nv, int m, int prec) { return rec_stride(nv * ncoef_h(dim, m), elem_bytes(prec, m)); }

struct WsLayout {
    size_t status, o0[2], ord[MAXN + 1], ustage, total;
};

WsLayout ws_layout(const dolinc_mesh *m, const dolinc_scheme *s)
{
    WsLayout L{};
    const size_t nc = (size_t)m->h.n_cells;
    size_t o = 0;
    L.status = o;
    o += 256;
    for (int i = 0; i < 2; ++i) {
        L.o0[i] = o;
        o += al256(nc * stride_h(m->h.dim, s->nv, 0, s->precision) * elem_bytes(s->precision, 0));
    }
    L.ord[0] = L.o0[0];
    for (int mm = 1; mm <= MAXN; ++mm) {
        L.ord[mm] = o;
        if (mm <= s->n_diff) o += al256(nc * stride_h(m->h.dim, s->nv, mm, s->precision) * elem_bytes(s->precision, mm));
    }
    L.ustage = o;
    o += al256(nc * s->nv * sizeof(double));
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
    a.flags = s->limiter == DOLINC_LIMIT_ENO3_FLAGGED ? m->flags : nullptr;
    a.eno_all = s->limiter == DOLINC_LIMIT_ENO3_ALL;
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
        timed(m, mm, st, [&] { p->diff(m->d, mm, B(ws, mm == 1 ? o0off : L.ord[mm - 1]), B(ws, L.ord[mm]), t, st); });
}

dolinc_status launch_check()
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(DOLINC_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return DOLINC_OK;
}

}  // namespace

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
    cudaGetDevice(&m->device);
    const HostMesh &h = m->h;
    const int64_t nc = h.n_cells, nf = h.n_faces, ns = h.n_slots;
    std::vector<int2> slot2(ns);
    std::vector<double> sk64(4 * ns), ck64(4 * nc), f64(8 * nf);
    std::vector<float> sk32(4 * ns), ck32(4 * nc), f32(8 * nf);
    for (int64_t s = 0; s < ns; ++s) {
        slot2[s] = make_int2(h.snb[s], (int)h.sword[s]);
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
    for (int64_t c = 0; c < nc; ++c) m->max_faces = std::max(m->max_faces, (int)(h.off[c + 1] - h.off[c]));
    dolinc_status st = DOLINC_OK;
    DevMesh &d = m->d;
    d.dim = h.dim;
    d.n_cells = (int)nc;
    d.n_faces = (int)nf;
    d.n_slots = (int)ns;
    if ((st = upload(m, off, &d.off)) || (st = upload(m, slot2, &d.slot2)) || (st = upload(m, sk64, &d.slotk64)) ||
        (st = upload(m, sk32, &d.slotk32)) || (st = upload(m, ck64, &d.cellk64)) ||
        (st = upload(m, ck32, &d.cellk32)) || (st = upload(m, f64, &d.face64)) || (st = upload(m, f32, &d.face32)) ||
        (st = upload(m, fo, &d.fo)) || (st = upload(m, fn, &d.fn)) || (st = upload(m, fe, &d.face_ext)) ||
        (st = upload(m, ff, &d.face_flip))) {
        delete m;
        return st;
    }
    *out = m;
    return DOLINC_OK;
}

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
    dolinc_status st = check_scheme(m, s);
    if (st) return st;
    if (!bytes) return fail(DOLINC_ERR_INVALID_ARG, "null bytes");
    *bytes = ws_layout(m, s).total;
    return DOLINC_OK;
}

dolinc_status dolinc_workspace_init(void *ws, size_t bytes, dolinc_stream stream)
{
    if (!ws || bytes < 256) return fail(DOLINC_ERR_INVALID_ARG, "workspace must hold at least 256 bytes");
    if (((uintptr_t)ws & 255) != 0) return fail(DOLINC_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    CU(cudaMemsetAsync(ws, 0, 256, reinterpret_cast<cudaStream_t>(stream)));
    return DOLINC_OK;
}

dolinc_status dolinc_diff_layout(const dolinc_mesh *m, const dolinc_scheme *s, int order, int64_t *offset,
                                 int *stride, int *eb, int64_t *total_bytes)
{
    dolinc_status st = check_scheme(m, s);
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
    const PathFns *p = path_for(m, s, needed_order(*s));
    if (!p) return fail(DOLINC_ERR_UNSUPPORTED, "no kernel for this (dim, nv, order, precision)");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    timed(m, DOLINC_KERNEL_PACK, cs, [&] { p->pack(m->d, u, B(ws, L.o0[0]), cs); });
    size_t o = 0;
    const void *prev = B(ws, L.o0[0]);
    for (int mm = 1; mm <= order; ++mm) {
        const int b = elem_bytes(s->precision, mm), sd = stride_h(m->h.dim, s->nv, mm, s->precision);
        timed(m, mm, cs, [&] { p->diff(m->d, mm, prev, B(diff, o), tune_for(m, s), cs); });
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
    timed(m, DOLINC_KERNEL_PACK, cs, [&] { p->pack(m->d, u, B(ws, L.o0[0]), cs); });
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
    timed(m, DOLINC_KERNEL_PACK, cs, [&] { p->pack(m->d, u, B(ws, L.o0[0]), cs); });
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
    timed(m, DOLINC_KERNEL_PACK, cs, [&] { p->pack(m->d, us, B(ws, L.o0[0]), cs); });
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

dolinc_status dolinc_rk_step(dolinc_mesh *m, const dolinc_scheme *s, double dt, double *u, void *ws,
                             size_t ws_bytes, dolinc_stream stream)
{
    static const double A[3] = {0.0, 0.75, 1.0 / 3.0}, Bc[3] = {1.0, 0.25, 2.0 / 3.0};
    dolinc_status st = check_scheme(m, s);
    if (st) return st;
    WsLayout L;
    if ((st = check_ws(m, s, ws, ws_bytes, L))) return st;
    if (!u) return fail(DOLINC_ERR_INVALID_ARG, "null field");
    const PathFns *p = path_for(m, s, needed_order(*s));
    if (!p) return fail(DOLINC_ERR_UNSUPPORTED, "no kernel for this (dim, nv, order, precision)");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    double *ust = reinterpret_cast<double *>(B(ws, L.ustage));
    const Tune tn = tune_for(m, s);
    timed(m, DOLINC_KERNEL_PACK, cs, [&] { p->pack(m->d, u, B(ws, L.o0[0]), cs); });
    int cur = 0;
    for (int sg = 0; sg < 3; ++sg) {
        run_diffs(m, p, ws, L, L.o0[cur], s->n_diff, tn, cs);
        StageArgs a = base_args(m, s, ws, L, L.o0[cur]);
        a.mode = 1;
        a.u0 = u;
        a.us = sg == 0 ? u : ust;
        a.out = sg == 2 ? u : ust;
        a.A = A[sg];
        a.B = Bc[sg];
        a.dt = dt;
        a.o0_next = sg == 2 ? nullptr : B(ws, L.o0[1 - cur]);
        timed(m, DOLINC_KERNEL_STAGE, cs, [&] { p->stage(m->d, a, tune_for(m, s), cs); });
        cur = 1 - cur;
    }
    return launch_check();
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
        p->pack(m->d, u, B(ws, L.o0[0]), cs);
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
        const int lpcs[3] = {1, 4, 8}, blocks[3] = {64, 128, 256};
        double bd = 1e30, bs = 1e30;
        for (int li = 0; li < 3; ++li)
            for (int bi = 0; bi < 3; ++bi) {
                Tune t;
                t.diff_lpc = t.stage_lpc = lpcs[li];
                t.diff_block = t.stage_block = blocks[bi];
                double td = time_it([&] {
                    for (int mm = 1; mm <= s->n_diff; ++mm)
                        p->diff(m->d, mm, B(ws, mm == 1 ? L.o0[0] : L.ord[mm - 1]), B(ws, L.ord[mm]), t, cs);
                });
                StageArgs a = base_args(m, s, ws, L, L.o0[0]);
                a.mode = 0;
                a.out = reinterpret_cast<double *>(B(ws, L.ustage));
                double tsg = time_it([&] { p->stage(m->d, a, t, cs); });
                if (td < bd) bd = td, best.diff_lpc = t.diff_lpc, best.diff_block = t.diff_block;
                if (tsg < bs) bs = tsg, best.stage_lpc = t.stage_lpc, best.stage_block = t.stage_block;
            }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        m->prof = prof;
        best_diff = bd;
        best_stage = bs;
        CU(cudaMemsetAsync(B(ws, L.status), 0, 256, cs));   // the timing runs may have flagged garbage
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

dolinc_status dolinc_set_tuning(dolinc_mesh *m, const dolinc_scheme *s, const dolinc_tuning *t)
{
    dolinc_status st = check_scheme(m, s);
    if (st) return st;
    if (!t) return fail(DOLINC_ERR_INVALID_ARG, "null tuning");
    auto ok_l = [](int l) { return l == 1 || l == 4 || l == 8; };
    auto ok_b = [](int b) { return b >= 32 && b <= 256 && b % 32 == 0; };
    if (!ok_l(t->diff_lanes) || !ok_l(t->stage_lanes) || !ok_b(t->diff_block) || !ok_b(t->stage_block))
        return fail(DOLINC_ERR_INVALID_ARG, "lanes must be 1, 4 or 8 and blocks a multiple of 32 in 32..256");
    Tune x;
    x.diff_lpc = t->diff_lanes;
    x.diff_block = t->diff_block;
    x.stage_lpc = t->stage_lanes;
    x.stage_block = t->stage_block;
    m->tuned[scheme_key(m, s)] = x;
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
    CU(cudaMemsetAsync(ws, 0, sizeof h, cs));
    CU(cudaStreamSynchronize(cs));
    if (h & 2u) return fail(DOLINC_ERR_DEVICE_TIMEOUT, "a device-side wait gave up");
    if (h & 1u) return fail(DOLINC_ERR_NONFINITE, "a stage produced NaN or Inf");
    return DOLINC_OK;
}

}  // extern "C"
