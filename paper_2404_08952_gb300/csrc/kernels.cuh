// DOLINC stage kernels for sm_103a.  Each cell gathers over its own face slots, so no
// kernel uses atomics on field data.
//
//   k_pack    FP64 cell averages [v][c]  ->  order-0 record (bulk precision, per cell)
//   k_diff    order m-1 -> order m differential (Sec 2.3), the Gauss step on the
//             polynomial coefficients:  p_m = w_c (S.d) p_{m-1,c} + sum_f k_f (S.d) p_{m-1,nb}
//   k_bnd_grad  Dirichlet / Neumann faces' correction of the first-order record (Sec 2.6)
//   k_stage   per cell and face: contract both cells' differentials with d, invert +
//             reconstruct both orientations (Secs 2.3-2.4), numerical flux (Sec 3),
//             residual, then the stage epilogue: the SSP-RK3 combination in FP64, or
//             below FP64 the increment form, and the next order-0 record.
//             A face is evaluated identically from its two cells (canonical
//             owner -> neighbour orientation, same operands, same order), so the two
//             contributions cancel exactly in the sum over cells.
//   k_flux + k_gather  the same stage face-centric: every face evaluated once into a
//             flux array, then each cell sums its signed fluxes in slot order
//   k_stage_tile / k_diff_tile  block-tiled variants (records staged in shared memory)
//   k_batch_stage  one cooperative launch per stage over many concatenated meshes
//   k_faces   face states written in the caller's face order (diagnostic entry point)
#pragma once
#include "common.cuh"
#include "device_mesh.hpp"
#include "tma.cuh"

namespace dol {

enum { PREC_F64 = 0, PREC_F32 = 1, PREC_BF16 = 2 };

template <int PREC> struct PrecT;
template <> struct PrecT<PREC_F64> { using R = double; using T0 = double; using TH = double; };
template <> struct PrecT<PREC_F32> { using R = float; using T0 = float; using TH = float; };
template <> struct PrecT<PREC_BF16> { using R = float; using T0 = float; using TH = __nv_bfloat16; };

// storage type of order m
template <int PREC, int M> struct OrdT { using T = typename std::conditional<(M >= 2), typename PrecT<PREC>::TH, typename PrecT<PREC>::T0>::type; };

template <int DIM, int NV, int M, int PREC>
DOL_HD constexpr int ord_stride() { return rec_stride(NV * ncoef(DIM, M), (int)sizeof(typename OrdT<PREC, M>::T)); }

template <class R> struct Geo;
template <> struct Geo<double> {
    static __device__ __forceinline__ const double *slotk(const DevMesh &m) { return m.slotk64; }
    static __device__ __forceinline__ const double *cellk(const DevMesh &m) { return m.cellk64; }
    static __device__ __forceinline__ const double *face(const DevMesh &m) { return m.face64; }
    static __device__ __forceinline__ int nb_of(double w) { return (int)__double_as_longlong(w); }
    static __device__ __forceinline__ const double *bval(const DevMesh &m) { return m.bval64; }
    static __device__ __forceinline__ const double *bdelta(const DevMesh &m) { return m.bdelta64; }
    static __device__ __forceinline__ const double *fdelta(const DevMesh &m) { return m.fdelta64; }
};
template <> struct Geo<float> {
    static __device__ __forceinline__ const float *slotk(const DevMesh &m) { return m.slotk32; }
    static __device__ __forceinline__ const float *cellk(const DevMesh &m) { return m.cellk32; }
    static __device__ __forceinline__ const float *face(const DevMesh &m) { return m.face32; }
    static __device__ __forceinline__ int nb_of(float w) { return __float_as_int(w); }
    static __device__ __forceinline__ const float *bval(const DevMesh &m) { return m.bval32; }
    static __device__ __forceinline__ const float *bdelta(const DevMesh &m) { return m.bdelta32; }
    static __device__ __forceinline__ const float *fdelta(const DevMesh &m) { return m.fdelta32; }
};

// Slot range [s0, s1) of cell c: a fixed stride when every cell has the same number of
// slots (tetrahedra, hexahedra, triangles, quads), else the CSR offsets.
__device__ __forceinline__ void slot_range(const DevMesh &mesh, int c, int &s0, int &s1)
{
    if (mesh.uniform_slots > 0) {
        s0 = c * mesh.uniform_slots;
        s1 = s0 + mesh.uniform_slots;
    } else {
        s0 = __ldg(mesh.off + c);
        s1 = __ldg(mesh.off + c + 1);
    }
}

// State on boundary face f of a cell whose state is U (Sec 2.6): a Dirichlet face
// takes its prescribed value, a Neumann face U + q delta (q the outward normal
// gradient, delta the centroid-to-face normal distance); other faces keep U.
template <int NV, class R>
__device__ __forceinline__ void boundary_state(const DevMesh &mesh, int f, R *U)
{
    if (!mesh.bidx) return;
    const int b = __ldg(mesh.bidx + f);
    if (b < 0) return;
    const R *val = Geo<R>::bval(mesh);
    const bool dirichlet = __ldg(mesh.bkind + b) == 2;
    const R delta = __ldg(Geo<R>::bdelta(mesh) + b);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const R x = __ldg(val + (long long)v * mesh.n_bv + b);
        U[v] = dirichlet ? x : U[v] + x * delta;
    }
}

// 8 values of a 32-byte aligned record: 256-bit loads from global memory, else two ld4
template <class R, bool LDG = true> __device__ __forceinline__ void ld8(const R *p, R *x);

template <class R, bool LDG = true> __device__ __forceinline__ void ld4(const R *p, R &a, R &b, R &c, R &d)
{
    if constexpr (sizeof(R) == 4) {
        float4 v = ldv<LDG>(reinterpret_cast<const float4 *>(p));
        a = v.x, b = v.y, c = v.z, d = v.w;
    } else {
        double2 v0 = ldv<LDG>(reinterpret_cast<const double2 *>(p));
        double2 v1 = ldv<LDG>(reinterpret_cast<const double2 *>(p) + 1);
        a = v0.x, b = v0.y, c = v1.x, d = v1.y;
    }
}

template <class R, bool LDG> __device__ __forceinline__ void ld8(const R *p, R *x)
{
    if constexpr (LDG) {
        unsigned w[8];
#pragma unroll
        for (int h = 0; h < (int)sizeof(R); h += 4) {
            ldg32(p + 8 * h / (int)sizeof(R), w);
            const R *e = reinterpret_cast<const R *>(w);
#pragma unroll
            for (int j = 0; j < 32 / (int)sizeof(R); ++j) x[8 * h / (int)sizeof(R) + j] = e[j];
        }
    } else {
        ld4<R, false>(p, x[0], x[1], x[2], x[3]);
        ld4<R, false>(p + 4, x[4], x[5], x[6], x[7]);
    }
}

// ------------------------------------------------------------------ pack
// copy (may be null): also written with u, e.g. a device copy of a state that u reads
// from mapped host memory
template <int NV, int PREC>
__global__ void __launch_bounds__(256) k_pack(int n, const double *__restrict__ u, typename PrecT<PREC>::T0 *o0,
                                              double *__restrict__ copy)
{
    using R = typename PrecT<PREC>::R;
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    double x[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) x[i] = u[(long long)i * n + c];
    if (copy) {
#pragma unroll
        for (int i = 0; i < NV; ++i) copy[(long long)i * n + c] = x[i];
    }
    R v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = (R)x[i];
    store_rec<typename PrecT<PREC>::T0, NV, rec_stride(NV, (int)sizeof(typename PrecT<PREC>::T0))>(o0, c, v);
}

// ------------------------------------------------------------------ differential pass
// LPC lanes per cell: lane l gathers slots l, l+LPC, ... (lane 0 adds the cell's own
// term), the group sums by recursive halving and each lane stores its slice of the
// output record.  LPC = 1 is one thread per cell.
DOL_HD constexpr int round_up(int n, int q) { return ((n + q - 1) / q) * q; }
// slots gathered per batch, by the size of the input record (registers held per slot)
DOL_HD constexpr int diff_batch(int rec_values) { return rec_values <= 8 ? 4 : (rec_values <= 16 ? 2 : 1); }

// One differential pass over a group of nt threads (thread t of the group, global
// thread index gt of the pass; for LPC = 1 the group's cells start at c0 and its
// output records are staged in smo and written by thread 0 with one bulk copy).
template <int DIM, int NV, int M, int PREC, int LPC, int UBF = 0>
__device__ __forceinline__ void diff_cells(const DevMesh &mesh, const void *__restrict__ in_v, void *__restrict__ out_v,
                                           long long gt, int t, int nt, long long c0, unsigned char *smo)
{
    using R = typename PrecT<PREC>::R;
    using TI = typename OrdT<PREC, M - 1>::T;
    using TO = typename OrdT<PREC, M>::T;
    constexpr int CI = ncoef(DIM, M - 1), CO = ncoef(DIM, M);
    constexpr int SI = ord_stride<DIM, NV, M - 1, PREC>(), SO = ord_stride<DIM, NV, M, PREC>();
    const TI *in = static_cast<const TI *>(in_v);
    TO *out = static_cast<TO *>(out_v);
    const int c = (int)(gt / LPC), l = (int)(gt % LPC);
    const bool valid = c < mesh.n_cells;
    constexpr int VO = 16 / (int)sizeof(TO);
    constexpr int P = (LPC == 1) ? NV * CO : round_up(SO, LPC * VO);   // SO >= NV * CO
    R acc[P];
#pragma unroll
    for (int i = 0; i < P; ++i) acc[i] = (R)0;
    if (valid) {
        int s0, s1;
        slot_range(mesh, c, s0, s1);
        // Slots in batches of UB, whose neighbour records are all requested before the
        // first is used.  The slot records of the first batch are requested before the
        // cell's own term is summed; with batches of one or two slots (large records,
        // few registers to spare for a batch) those of the next batch are requested
        // before the current batch is summed.  The sums keep the order own term, then
        // slots in order.
        constexpr int UB = UBF > 0 ? UBF : diff_batch(NV * CI);   // UBF: a batch size forced by the caller
        constexpr bool PREFETCH = UB <= 2;
        R kx[UB], ky[UB], kz[UB];
        int nbv[UB];
        bool ok[UB];
        auto load_k = [&](int s) {
            R kb[UB];
#pragma unroll
            for (int u = 0; u < UB; ++u) {
                ok[u] = s + u * LPC < s1;
                kb[u] = kx[u] = ky[u] = kz[u] = (R)0;
            }
            if constexpr (LPC == 1 && UB >= 4 && UB % 2 == 0 && sizeof(R) == 4) {
                // two consecutive 16-byte slot records starting at an even slot are one
                // aligned 32-byte load
#pragma unroll
                for (int u = 0; u < UB; u += 2) {
                    const int su = s + u;
                    if (ok[u + 1] && (su & 1) == 0) {
                        R k8[8];
                        ld8<R>(Geo<R>::slotk(mesh) + 4ll * su, k8);
                        kx[u] = k8[0], ky[u] = k8[1], kz[u] = k8[2], kb[u] = k8[3];
                        kx[u + 1] = k8[4], ky[u + 1] = k8[5], kz[u + 1] = k8[6], kb[u + 1] = k8[7];
                    } else {
                        if (ok[u]) ld4<R>(Geo<R>::slotk(mesh) + 4ll * su, kx[u], ky[u], kz[u], kb[u]);
                        if (ok[u + 1])
                            ld4<R>(Geo<R>::slotk(mesh) + 4ll * (su + 1), kx[u + 1], ky[u + 1], kz[u + 1], kb[u + 1]);
                    }
                }
            } else {
#pragma unroll
                for (int u = 0; u < UB; ++u)
                    if (ok[u]) ld4<R>(Geo<R>::slotk(mesh) + 4ll * (s + u * LPC), kx[u], ky[u], kz[u], kb[u]);
            }
#pragma unroll
            for (int u = 0; u < UB; ++u) nbv[u] = Geo<R>::nb_of(kb[u]);
        };
        load_k(s0 + l);
        if (l == 0) {
            R x[NV * CI];
            R wx, wy, wz, iv;
            ld4<R>(Geo<R>::cellk(mesh) + 4ll * c, wx, wy, wz, iv);
            load_rec<TI, NV * CI, SI, R>(in, c, x);
            poly_mul_acc<DIM, NV, M, R>(acc, x, wx, wy, wz);
        }
        for (int s = s0 + l; s < s1; s += LPC * UB) {
            R xs[UB][NV * CI];
#pragma unroll
            for (int u = 0; u < UB; ++u)
                if (ok[u]) load_rec<TI, NV * CI, SI, R>(in, nbv[u], xs[u]);
            R cx[UB], cy[UB], cz[UB];
            bool cok[UB];
#pragma unroll
            for (int u = 0; u < UB; ++u) cx[u] = kx[u], cy[u] = ky[u], cz[u] = kz[u], cok[u] = ok[u];
            if constexpr (PREFETCH) load_k(s + LPC * UB);
#pragma unroll
            for (int u = 0; u < UB; ++u)
                if (cok[u]) poly_mul_acc<DIM, NV, M, R>(acc, xs[u], cx[u], cy[u], cz[u]);
            if constexpr (!PREFETCH) load_k(s + LPC * UB);
        }
    }
    if constexpr (LPC == 1) {
        constexpr unsigned RBO = SO * (unsigned)sizeof(TO);
        if constexpr (RBO % 16 == 0) {
            // the block's records are contiguous: stage them in shared memory and write
            // them with one bulk copy
            if (valid) store_rec_smem<TO, NV * CO, SO, R>(smo, t, acc);
            fence_proxy_async_smem();
            __syncthreads();
            if (t == 0 && c0 < mesh.n_cells) {
                const unsigned n = (unsigned)min((long long)nt, (long long)mesh.n_cells - c0);
                bulk_s2g_wait(out + c0 * SO, smo, n * RBO);
            }
        } else {
            if (valid) store_rec<TO, NV * CO, SO, R>(out, c, acc);
        }
    } else {
        group_reduce_scatter<P, LPC, R>(acc, l);
        if (!valid) return;
        constexpr int B = P / LPC;                 // elements this lane owns
        const int e0 = l * B;
        TO *rec = out + (long long)c * SO;
        if constexpr ((B * (int)sizeof(TO)) % 16 == 0 && (SO * (int)sizeof(TO)) % 16 == 0) {
#pragma unroll
            for (int i = 0; i < B / VO; ++i) {
                if (e0 + i * VO < SO) {
                    uint4 q;
                    TO *e = reinterpret_cast<TO *>(&q);
#pragma unroll
                    for (int j = 0; j < VO; ++j)
                        e[j] = (e0 + i * VO + j < NV * CO) ? to_store<TO, R>(acc[i * VO + j]) : to_store<TO, R>((R)0);
                    *reinterpret_cast<uint4 *>(rec + e0 + i * VO) = q;
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < B; ++i)
                if (e0 + i < NV * CO) rec[e0 + i] = to_store<TO, R>(acc[i]);
        }
    }
}


template <int DIM, int NV, int M, int PREC, int LPC>
__global__ void __launch_bounds__(256) k_diff(DevMesh mesh, const void *__restrict__ in_v, void *__restrict__ out_v)
{
    extern __shared__ __align__(16) unsigned char smo[];
    diff_cells<DIM, NV, M, PREC, LPC>(mesh, in_v, out_v, (long long)blockIdx.x * blockDim.x + threadIdx.x,
                                      threadIdx.x, blockDim.x, (long long)blockIdx.x * blockDim.x, smo);
}

// Two differential passes in one launch over the same cells: the first CB threads of
// a block gather order MA (inA -> outA), the next CB threads order 1 (inB -> outB),
// for the block's CB cells.  Both halves read the cells' slot and cell weights, which
// the second half finds in L1: one read of the Gauss weights for two passes (the order
// a stage does not read, with the next stage's first order).  Each half is the
// one-thread-per-cell pass (diff_cells), so every output is bit-identical to it.
template <int DIM, int NV, int MA, int PREC, int CB, int MINB = 1>
__global__ void __launch_bounds__(2 * CB, MINB) k_diff_dual(DevMesh mesh, const void *__restrict__ inA, void *__restrict__ outA,
                                                      const void *__restrict__ inB, void *__restrict__ outB)
{
    // both halves stage their records for a bulk copy, i.e. pass one __syncthreads
    static_assert((ord_stride<DIM, NV, MA, PREC>() * sizeof(typename OrdT<PREC, MA>::T)) % 16 == 0 &&
                      (ord_stride<DIM, NV, 1, PREC>() * sizeof(typename OrdT<PREC, 1>::T)) % 16 == 0,
                  "records of whole 16-byte chunks in both passes");
    extern __shared__ __align__(16) unsigned char smo[];
    const int t = threadIdx.x % CB;
    const long long c0 = (long long)blockIdx.x * CB;
    // the order-MA half gathers one slot per batch (the other half's loads are in flight
    // meanwhile): fewer registers, the same sums in the same order
    if (threadIdx.x < CB)
        diff_cells<DIM, NV, MA, PREC, 1, 1>(mesh, inA, outA, c0 + t, t, CB, c0, smo);
    else
        diff_cells<DIM, NV, 1, PREC, 1>(mesh, inB, outB, c0 + t, t, CB, c0,
                                        smo + (size_t)CB * ord_stride<DIM, NV, MA, PREC>() *
                                                  sizeof(typename OrdT<PREC, MA>::T));
}

// ------------------------------------------------------------------ stage
struct StageArgs {
    const void *ord[MAXN + 1];   // order records 0..NS (order 0 = bulk copy of the stage input)
    void *o0_next;               // order-0 record of the stage output (may be null)
    const double *u0, *us;       // FP64 step start and stage input [v][c]
    double *out;                 // FP64 output [v][c]: residual (mode 0), stage value (mode 1),
                                 // or the step's new state (mode 2, last stage)
    double A, B, dt;             // out = A u0 + B (us + dt R)
    float *dacc;                 // mode 2: increment accumulator D [v][c] (bulk precision)
    const void *rec_start;       // mode 2: order-0 record of the step's start state
    int rk;                      // mode 2: SSP-RK3 stage index 0, 1, 2
    void *face_flux;             // face-centric stage: per-face fluxes [v][face] (bulk precision)
    unsigned *status;            // bit 0: non-finite output
    int k, r, mode, flux;
    double gamma, adv[3];
    const uint8_t *flags;        // faces touching a flagged cell are limited (null: none)
    int all_mode;                // limit of every face: LIM_NONE, LIM_ENO3 or LIM_WENO5
    int flag_mode;               // limit of flagged faces: LIM_ENO3, LIM_FIRST_ORDER or LIM_WENO5
};

// Face limit: none, ENO3-DOLINC, first-order upwind (each side's own cell average),
// or WENO5-DOLINC
enum { LIM_NONE = 0, LIM_ENO3 = 1, LIM_FIRST_ORDER = 2, LIM_WENO5 = 3 };

__device__ __forceinline__ int face_limit(const StageArgs &a, bool flagged)
{
    return a.all_mode != LIM_NONE ? a.all_mode : (flagged ? a.flag_mode : LIM_NONE);
}

// Where a kernel reads cell records and face records from.  GlobalSrc: device memory
// through the read-only path.  TileSrc (k_stage_tile): the block's own cells and the
// faces they own were staged in shared memory; other cells/faces come from global.
template <int DIM, int NV, int PREC> struct GlobalSrc {
    using R = typename PrecT<PREC>::R;
    static constexpr bool LDG = true;
    const StageArgs &a;
    const DevMesh &mesh;
    template <int M> __device__ __forceinline__ const typename OrdT<PREC, M>::T *rec(int X) const
    {
        return static_cast<const typename OrdT<PREC, M>::T *>(a.ord[M]) + (long long)X * ord_stride<DIM, NV, M, PREC>();
    }
    __device__ __forceinline__ const R *face(int f) const { return Geo<R>::face(mesh) + 8ll * f; }
};

template <int DIM, int NV, int NS, int PREC> struct TileSrc {
    using R = typename PrecT<PREC>::R;
    static constexpr bool LDG = false;
    const StageArgs &a;
    const DevMesh &mesh;
    const unsigned char *sm;          // staged records of orders 0..NS, then faces
    int t0, nt, f_lo, f_hi;
    unsigned off[NS + 2];             // byte offsets of order m (m = 0..NS) and of the faces
    template <int M> __device__ __forceinline__ const typename OrdT<PREC, M>::T *rec(int X) const
    {
        using T = typename OrdT<PREC, M>::T;
        constexpr int S = ord_stride<DIM, NV, M, PREC>();
        const unsigned i = (unsigned)(X - t0);
        if (i < (unsigned)nt) return reinterpret_cast<const T *>(sm + off[M]) + (long long)i * S;
        return static_cast<const T *>(a.ord[M]) + (long long)X * S;
    }
    __device__ __forceinline__ const R *face(int f) const
    {
        if (f >= f_lo && f < f_hi) return reinterpret_cast<const R *>(sm + off[NS + 1]) + 8ll * (f - f_lo);
        return Geo<R>::face(mesh) + 8ll * f;
    }
};

// phi^(m) of every variable of cell X along the monomials of d (m = 0..NS)
template <int DIM, int NV, int NS, int PREC, int M, class Src>
__device__ __forceinline__ void contract_order(const Src &src, int X, const typename PrecT<PREC>::R *mono,
                                               typename PrecT<PREC>::R (*ph)[NS + 1])
{
    using R = typename PrecT<PREC>::R;
    using T = typename OrdT<PREC, M>::T;
    constexpr int C = ncoef(DIM, M);
    R rec[NV * C];
    load_rec<T, NV * C, ord_stride<DIM, NV, M, PREC>(), R, Src::LDG>(src.template rec<M>(X), 0, rec);
    constexpr int mo = ncum(DIM, M - 1);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        R s = (R)0;
#pragma unroll
        for (int q = 0; q < C; ++q) s = fma(rec[v * C + q], mono[mo + q], s);
        ph[v][M] = s * (R)(1 << M);
    }
}

template <int DIM, int NV, int NS, int PREC, class Src>
__device__ __forceinline__ void contract_cell(const Src &src, int X, const typename PrecT<PREC>::R *mono,
                                              typename PrecT<PREC>::R (*ph)[NS + 1])
{
    using R = typename PrecT<PREC>::R;
    {
        R rec[NV];
        load_rec<typename PrecT<PREC>::T0, NV, ord_stride<DIM, NV, 0, PREC>(), R, Src::LDG>(src.template rec<0>(X),
                                                                                             0, rec);
#pragma unroll
        for (int v = 0; v < NV; ++v) ph[v][0] = rec[v];
    }
    if constexpr (NS >= 1) contract_order<DIM, NV, NS, PREC, 1>(src, X, mono, ph);
    if constexpr (NS >= 2) contract_order<DIM, NV, NS, PREC, 2>(src, X, mono, ph);
    if constexpr (NS >= 3) contract_order<DIM, NV, NS, PREC, 3>(src, X, mono, ph);
    if constexpr (NS >= 4) contract_order<DIM, NV, NS, PREC, 4>(src, X, mono, ph);
}

template <int DIM, int NV, int NS, int PREC>
__device__ __forceinline__ void contract_cell(const StageArgs &a, int X, const typename PrecT<PREC>::R *mono,
                                              typename PrecT<PREC>::R (*ph)[NS + 1], const DevMesh &mesh)
{
    GlobalSrc<DIM, NV, PREC> src{a, mesh};
    contract_cell<DIM, NV, NS, PREC>(src, X, mono, ph);
}

// ENO3-DOLINC value of one variable (Sec 2.4): far values n = -2..2 by Eq diffDLC, the
// paper's non-uniform indicators, then the k = 3 weights of the chosen stencil.
template <int NS, class R>
__device__ __forceinline__ R eno3_value(R g, const R *p0, const R *p1)
{
    static_assert(NS >= 2, "ENO3 needs second-order differentials");
    // phi_{-1}^(m) (m = 0, 1), phi_{-2}, phi_2
    R gi = (R)1 / g;
    R m1_0 = gi * (p1[0] - p0[1] - ((R)1 - g) * p0[0]);
    R m1_1 = gi * (p1[1] - p0[2] - ((R)1 - g) * p0[1]);
    R m2 = gi * (p0[0] - gi * m1_1 - ((R)1 - g) * m1_0);
    R p2 = g * p0[0] + g * p1[1] + ((R)1 - g) * p1[0];
    R d2l = g * (p0[0] - m1_0), d2r = p1[0] - p0[0];
    R dL = g * g * (p0[0] - ((R)1 + g) * m1_0 + g * m2);
    R dC = p1[0] - ((R)1 + g) * p0[0] + g * m1_0;
    R dR = (p2 - ((R)1 + g) * p1[0] + g * p0[0]) * gi * gi;
    int r = (fabs(d2l) <= fabs(d2r)) ? (fabs(dL) < fabs(dC) ? 2 : 1) : (fabs(dR) < fabs(dC) ? 0 : 1);
    // k = 3 weights on the geometric cells (closed forms of Eq coeff)
    R g2 = g * g, G2 = (R)1 + g, G3 = (R)1 + g + g2;
    if (r == 1) return (-g2 * g * m1_0 + g * ((R)1 + (R)2 * g + (R)2 * g2) * p0[0]) / (G2 * G3) + p1[0] / G3;
    if (r == 0) return (g2 * p0[0]) / G3 + ((g2 + (R)2 * g + (R)2) * p1[0] - p2) / (G2 * G3);
    return (g2 * g * m2) / G3 + (-g * (g2 * g + (R)3 * g2 + (R)2 * g + (R)1) * m1_0 +
                                 ((R)3 * g2 * g + (R)4 * g2 + (R)3 * g + (R)1) * p0[0]) / (G2 * G3);
}

// WENO5-DOLINC value of one variable (Sec 2.4: the fixed DOLINC stencils plus stencil
// weights).  The three 3-cell candidates on the geometric cells (closed forms of Eq
// coeff) are weighted by a_r = d_r / (1e-6 + beta_r)^2 (Jiang-Shu), with linear
// weights d_r that reproduce the 5-cell stencil (5,2):
//   d_2 = g^6 / (H G5),  d_0 = G3 / (H G5),  d_1 = g^2 G2 G3 / (H G5),
// G_n = 1 + g + .. + g^(n-1), H = 1 + g^2, and smoothness
//   beta_r = b_r^2 - b_r c_r + (4/3) c_r^2,
// b_r, c_r the slope at the upwind face and the curvature of the candidate's quadratic
// (the derivative of the cubic through its primitive) in units of the upwind cell,
// linear in the candidate's three values.  g = 1 gives the classical WENO5.
template <int NS, class R>
__device__ __forceinline__ R weno5_value(R g, const R *p0, const R *p1)
{
    static_assert(NS >= 2, "WENO5 needs second-order differentials");
    R gi = (R)1 / g;
    // far values phi_{-1}, phi_{-2}, phi_2 by Eq diffDLC (as for ENO3)
    R m1 = gi * (p1[0] - p0[1] - ((R)1 - g) * p0[0]);
    R m1_1 = gi * (p1[1] - p0[2] - ((R)1 - g) * p0[1]);
    R m2 = gi * (p0[0] - gi * m1_1 - ((R)1 - g) * m1);
    R q2f = g * p0[0] + g * p1[1] + ((R)1 - g) * p1[0];
    const R f0 = p0[0], f1 = p1[0];
    const R g2 = g * g, g3 = g2 * g;
    const R G2 = (R)1 + g, G3 = (R)1 + g + g2;
    const R D = G2 * G3, iD = (R)1 / D, iG3 = (R)1 / G3;
    // candidates (cells i..i+2, i-1..i+1, i-2..i)
    const R c0 = g2 * f0 * iG3 + ((g2 + (R)2 * g + (R)2) * f1 - q2f) * iD;
    const R c1 = (-g3 * m1 + g * ((R)1 + (R)2 * g + (R)2 * g2) * f0) * iD + f1 * iG3;
    const R c2 = g3 * m2 * iG3 + (-g * (g3 + (R)3 * g2 + (R)2 * g + (R)1) * m1 + ((R)3 * g3 + (R)4 * g2 + (R)3 * g + (R)1) * f0) * iD;
    // smoothness
    const R b0 = (R)2 * iD * (-g * (g + (R)2) * f0 + (g3 + (R)2 * g2 + g - (R)1) * gi * f1 - (g - (R)1) * gi * q2f);
    const R k0 = (R)6 * iD * (f0 - G2 * gi * f1 + gi * q2f);
    const R b1 = (R)2 * iD * (-g2 * (g - (R)1) * m1 + (g3 - g2 - (R)2 * g - (R)1) * f0 + ((R)2 * g + (R)1) * f1);
    const R k1 = (R)6 * g * iD * (g * m1 - G2 * f0 + f1);
    const R b2 = (R)2 * g * iD * (g2 * ((R)2 * g + (R)1) * m2 - ((R)2 * g3 + (R)4 * g2 + (R)2 * g + (R)1) * m1 +
                                  ((R)3 * g2 + (R)2 * g + (R)1) * f0);
    const R k2 = (R)6 * g3 * iD * (g * m2 - G2 * m1 + f0);
    const R be0 = b0 * b0 - b0 * k0 + (R)(4.0 / 3.0) * k0 * k0;
    const R be1 = b1 * b1 - b1 * k1 + (R)(4.0 / 3.0) * k1 * k1;
    const R be2 = b2 * b2 - b2 * k2 + (R)(4.0 / 3.0) * k2 * k2;
    // linear weights (common factor 1 / (H G5) cancels in the normalisation)
    const R d0 = G3, d1 = g2 * G2 * G3, d2 = g3 * g3;
    const R e0 = (R)1e-6 + be0, e1 = (R)1e-6 + be1, e2 = (R)1e-6 + be2;
    const R a0 = d0 / (e0 * e0), a1 = d1 / (e1 * e1), a2 = d2 / (e2 * e2);
    return (a0 * c0 + a1 * c1 + a2 * c2) / (a0 + a1 + a2);
}

// Both face states (or the upwind one only for linear advection) of face record fr.
template <int DIM, int NV, int NS, int PREC, bool UPWIND_ONLY, class Src>
__device__ __forceinline__ void face_states_dolinc(const StageArgs &a, const Src &src,
                                                   const typename PrecT<PREC>::R *fr, int P, int N, int lim,
                                                   typename PrecT<PREC>::R *UL, typename PrecT<PREC>::R *UR,
                                                   bool want_left)
{
    using R = typename PrecT<PREC>::R;
    if (lim == LIM_FIRST_ORDER) {
        constexpr int S0 = ord_stride<DIM, NV, 0, PREC>();
        load_rec<typename PrecT<PREC>::T0, NV, S0, R, Src::LDG>(src.template rec<0>(P), 0, UL);
        load_rec<typename PrecT<PREC>::T0, NV, S0, R, Src::LDG>(src.template rec<0>(N), 0, UR);
        return;
    }
    constexpr int NM = ncum(DIM, NS);
    R mono[NM];
    monomials<DIM, NS, R>(fr[0], fr[1], fr[2], mono);
    R phP[NV][NS + 1], phN[NV][NS + 1];
    contract_cell<DIM, NV, NS, PREC>(src, P, mono, phP);
    contract_cell<DIM, NV, NS, PREC>(src, N, mono, phN);
    const R g = fr[3];
    if constexpr (NS >= 2) {
        if (lim == LIM_ENO3) {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                R q0[3], q1[3];
#pragma unroll
                for (int m = 0; m < 3; ++m) { q0[m] = (m & 1) ? -phN[v][m] : phN[v][m]; q1[m] = (m & 1) ? -phP[v][m] : phP[v][m]; }
                if (!UPWIND_ONLY || want_left) UL[v] = eno3_value<NS, R>(g, phP[v], phN[v]);
                if (!UPWIND_ONLY || !want_left) UR[v] = eno3_value<NS, R>(rcp_bulk(g), q0, q1);
            }
            return;
        }
        if (lim == LIM_WENO5) {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                R q0[3], q1[3];
#pragma unroll
                for (int m = 0; m < 3; ++m) { q0[m] = (m & 1) ? -phN[v][m] : phN[v][m]; q1[m] = (m & 1) ? -phP[v][m] : phP[v][m]; }
                if (!UPWIND_ONLY || want_left) UL[v] = weno5_value<NS, R>(g, phP[v], phN[v]);
                if (!UPWIND_ONLY || !want_left) UR[v] = weno5_value<NS, R>((R)1 / g, q0, q1);
            }
            return;
        }
    }
    R W0[NS + 1], W1[NS + 1], V0[NS + 1], V1[NS + 1];
    if constexpr (!UPWIND_ONLY)
        dolinc_weights_both<NS, R>(a.k, a.r, g, W0, W1, V0, V1);     // both orientations, one reciprocal
    if (!UPWIND_ONLY || want_left) {
        if constexpr (UPWIND_ONLY) dolinc_weights<NS, R>(a.k, a.r, g, W0, W1);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            R s = (R)0;
#pragma unroll
            for (int m = 0; m <= NS; ++m) s = fma(W0[m], phP[v][m], fma(W1[m], phN[v][m], s));
            UL[v] = s;
        }
    }
    if (!UPWIND_ONLY || !want_left) {
        // neighbour upwind: d -> -d, g -> 1/g, phi^(m) -> (-1)^m phi^(m)
        if constexpr (UPWIND_ONLY) dolinc_weights<NS, R>(a.k, a.r, rcp_bulk(g), V0, V1);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            R s = (R)0;
#pragma unroll
            for (int m = 0; m <= NS; ++m) {
                R t = fma(V0[m], phN[v][m], V1[m] * phP[v][m]);
                s = (m & 1) ? s - t : s + t;
            }
            UR[v] = s;
        }
    }
}

// Skewness correction of the face states (mesh.fdelta non-null): the DOLINC value is
// that of the point x*_f of the centroid line; each orientation adds
// (x_f - x*_f) . T^(1) of its upwind cell to reach the face centroid.
template <int DIM, int NV, int PREC, class Src>
__device__ __forceinline__ void skew_shift(const Src &src, int f, int P, int N, typename PrecT<PREC>::R *UL,
                                           typename PrecT<PREC>::R *UR, bool doL, bool doR)
{
    using R = typename PrecT<PREC>::R;
    using T1 = typename OrdT<PREC, 1>::T;
    constexpr int C1 = ncoef(DIM, 1), S1 = ord_stride<DIM, NV, 1, PREC>();
    R dl[4];
    ld4<R>(Geo<R>::fdelta(src.mesh) + 4ll * f, dl[0], dl[1], dl[2], dl[3]);
    auto shift = [&](int X, R *U) {
        R r[NV * C1];
        load_rec<T1, NV * C1, S1, R, Src::LDG>(src.template rec<1>(X), 0, r);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            R t = U[v];
#pragma unroll
            for (int k = 0; k < DIM; ++k) t = fma(dl[k], r[v * C1 + k], t);
            U[v] = t;
        }
    };
    if (doL) shift(P, UL);
    if (doR) shift(N, UR);
}

// Face states of internal face f (face record fr): the DOLINC values, with the
// skewness correction when the mesh has it on (not on first-order fallback faces).
template <int DIM, int NV, int NS, int PREC, bool UPWIND_ONLY, class Src>
__device__ __forceinline__ void face_states(const StageArgs &a, const Src &src, const typename PrecT<PREC>::R *fr,
                                            int f, int P, int N, int lim, typename PrecT<PREC>::R *UL,
                                            typename PrecT<PREC>::R *UR, bool want_left)
{
    face_states_dolinc<DIM, NV, NS, PREC, UPWIND_ONLY>(a, src, fr, P, N, lim, UL, UR, want_left);
    if (Geo<typename PrecT<PREC>::R>::fdelta(src.mesh) && lim != LIM_FIRST_ORDER)
        skew_shift<DIM, NV, PREC>(src, f, P, N, UL, UR, !UPWIND_ONLY || want_left, !UPWIND_ONLY || !want_left);
}

template <int DIM, int NV, class R>
__device__ __forceinline__ void phys_flux(const StageArgs &a, const R *U, const R *fr, R *F)
{
    if constexpr (NV == 1) {
        if (a.flux == 0) {
            R an = (R)a.adv[0] * fr[4] + (R)a.adv[1] * fr[5] + (DIM == 3 ? (R)a.adv[2] * fr[6] : (R)0);
            F[0] = an * U[0];
        } else {
            R sg = fr[4] + fr[5] + (DIM == 3 ? fr[6] : (R)0);
            F[0] = (R)0.5 * U[0] * U[0] * sg;
        }
    } else {
        R un, c2;
        euler_phys<DIM, R>((R)a.gamma, U, fr[4], fr[5], fr[6], F, un, c2);
    }
}

// Numerical flux of the face of slot (nb, word) of cell c in the face's canonical
// owner -> neighbour orientation (a boundary slot: the flux of c's own state).  The
// operands and their order depend only on the face, not on which cell asks.
template <int DIM, int NV, int NS, int PREC, class Src>
__device__ __forceinline__ void canon_flux(const StageArgs &a, const Src &src, int c, int nb, unsigned word,
                                           bool own_flag, typename PrecT<PREC>::R *F)
{
    using R = typename PrecT<PREC>::R;
    const int f = (int)(word >> 2);
    const int side = word & 1;
    R fr[8];
    ld8<R, Src::LDG>(src.face(f), fr);
    if (word & 2) {
        // zero-gradient boundary (Sec 2.6): the auxiliary cell mirrors the cell value
        R U[NV];
        load_rec<typename PrecT<PREC>::T0, NV, ord_stride<DIM, NV, 0, PREC>(), R, Src::LDG>(src.template rec<0>(c), 0,
                                                                                            U);
        boundary_state<NV, R>(src.mesh, f, U);
        phys_flux<DIM, NV, R>(a, U, fr, F);
    } else {
        const int P = side ? nb : c, N = side ? c : nb;
        const int lim = face_limit(a, a.flags && (own_flag || a.flags[nb]));
        R UL[NV], UR[NV];
        if constexpr (NV == 1) {
            if (a.flux == 0) {
                R an = (R)a.adv[0] * fr[4] + (R)a.adv[1] * fr[5] + (DIM == 3 ? (R)a.adv[2] * fr[6] : (R)0);
                bool left = an >= (R)0;
                face_states<DIM, NV, NS, PREC, true>(a, src, fr, f, P, N, lim, UL, UR, left);
                F[0] = an * (left ? UL[0] : UR[0]);
            } else {
                face_states<DIM, NV, NS, PREC, false>(a, src, fr, f, P, N, lim, UL, UR, true);
                R sg = fr[4] + fr[5] + (DIM == 3 ? fr[6] : (R)0);
                R lam = (R)0.5 * (UL[0] + UR[0]) * sg;       // Roe speed of u^2/2 (1,..,1)
                R uu = lam >= (R)0 ? UL[0] : UR[0];
                F[0] = (R)0.5 * uu * uu * sg;
            }
        } else {
            face_states<DIM, NV, NS, PREC, false>(a, src, fr, f, P, N, lim, UL, UR, true);
            rusanov<DIM, R>((R)a.gamma, UL, UR, fr[4], fr[5], fr[6], fr[7], F);
        }
    }
}

// Numerical flux of the face in slot s of cell c, signed for c (+ into, - out of c).
template <int DIM, int NV, int NS, int PREC, class Src>
__device__ __forceinline__ void slot_flux(const DevMesh &mesh, const StageArgs &a, const Src &src, int c, int s,
                                          bool own_flag, typename PrecT<PREC>::R *F)
{
    const int2 sw = __ldg(mesh.slot2 + s);
    canon_flux<DIM, NV, NS, PREC>(a, src, c, sw.x, (unsigned)sw.y, own_flag, F);
    if (!(sw.y & 1)) {
#pragma unroll
        for (int v = 0; v < NV; ++v) F[v] = -F[v];
    }
}

// SSP-RK3 combination A u0 + B (us + dt R) with the increment dt R already formed in
// the bulk precision (R carries that precision's rounding anyway); FP64 then does only
// the state arithmetic: one add in stage 0 (A = 0, B = 1), add + mul + fma otherwise.
// NaN/Inf test on the bit pattern (integer pipe; keeps the scarce FP64 pipe free)
__device__ __forceinline__ bool nonfinite64(double x)
{
    return ((unsigned long long)__double_as_longlong(x) & 0x7ff0000000000000ull) == 0x7ff0000000000000ull;
}

template <class R>
__device__ __forceinline__ double stage_update(const StageArgs &a, long long i, R dtR)
{
    const double t = a.us[i] + (double)dtR;
    return a.A == 0.0 ? a.B * t : fma(a.B, t, a.A * a.u0[i]);
}

// Increment form of the SSP-RK3 step (mode 2, bulk precision below FP64).  With
// d_k = dt R(u_k) the three Shu-Osher stages expand to
//   u1 = u0 + D0,  u2 = u0 + D1,  u^{n+1} = u0 + (2/3)(D1 + d2),
//   D0 = d0,  D1 = (D0 + d1)/4,
// so the increment D of each cell is carried in the bulk precision between stages,
// the next stage's order-0 record is formed as (start record + D), and the FP64 state
// is touched once per step: one add in the last stage.
template <class R>
__device__ __forceinline__ bool nonfinite32(R x)
{
    return (__float_as_uint((float)x) & 0x7f800000u) == 0x7f800000u;
}

// Correctly rounded products and sums that the compiler may not fuse: the increment
// arithmetic is then the same in every stage kernel, whatever each one inlines.
__device__ __forceinline__ float mul_rn(float x, float y) { return __fmul_rn(x, y); }
__device__ __forceinline__ float add_rn(float x, float y) { return __fadd_rn(x, y); }

// Variable v of cell c; r = R_c (residual).  Returns true on NaN/Inf.
template <class R, class T0, int S0>
__device__ __forceinline__ bool incr_update(const StageArgs &a, int c, int v, long long n, R r, R dtr, T0 *nxt)
{
    const long long i = v * n + c;
    const R d = mul_rn(r, dtr);
    if (a.rk == 0) {
        a.dacc[i] = (float)d;
        const R u0 = (R)static_cast<const T0 *>(a.rec_start)[c * (long long)S0 + v];
        nxt[c * (long long)S0 + v] = (T0)add_rn(u0, d);
        return nonfinite32(d);
    }
    if (a.rk == 1) {
        const R D = mul_rn((R)0.25, add_rn((R)a.dacc[i], d));
        a.dacc[i] = (float)D;
        const R u0 = (R)static_cast<const T0 *>(a.rec_start)[c * (long long)S0 + v];
        nxt[c * (long long)S0 + v] = (T0)add_rn(u0, D);
        return nonfinite32(D);
    }
    const R D = mul_rn((R)(2.0 / 3.0), add_rn((R)a.dacc[i], d));
    const double o = __dadd_rn(a.u0[i], (double)D);
    a.out[i] = o;
    if (nxt) nxt[c * (long long)S0 + v] = (T0)(R)o;    // the next step's record (several steps per call)
    return nonfinite64(o);
}

// The same increment-form update for all NV variables of cell c (r[v] = R_c), with
// the step's start record read, and the next stage's record written, whole.
template <int NV, class R, class T0, int S0>
__device__ __forceinline__ bool incr_update_cell(const StageArgs &a, int c, long long n, const R *r, R dtr, T0 *nxt)
{
    bool bad = false;
    if (a.rk <= 1) {
        R u0[NV], nx[NV];
        load_rec<T0, NV, S0, R>(static_cast<const T0 *>(a.rec_start), c, u0);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const long long i = v * n + c;
            const R d = mul_rn(r[v], dtr);
            const R D = a.rk == 0 ? d : mul_rn((R)0.25, add_rn((R)a.dacc[i], d));
            a.dacc[i] = (float)D;
            nx[v] = add_rn(u0[v], D);
            bad |= nonfinite32(D);
        }
        store_rec<T0, NV, S0, R>(nxt, c, nx);
        return bad;
    }
    R nx[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const long long i = v * n + c;
        const R d = mul_rn(r[v], dtr);
        const R D = mul_rn((R)(2.0 / 3.0), add_rn((R)a.dacc[i], d));
        const double o = __dadd_rn(a.u0[i], (double)D);
        a.out[i] = o;
        nx[v] = (R)o;
        bad |= nonfinite64(o);
    }
    if (nxt) store_rec<T0, NV, S0, R>(nxt, c, nx);      // the next step's record (several steps per call)
    return bad;
}

// LPC lanes per cell: lane l evaluates slots l, l+LPC, ...; the group sums the signed
// fluxes by recursive halving and lane l then updates variables [l*B, (l+1)*B).
template <int DIM, int NV, int NS, int PREC, int LPC>
__global__ void __launch_bounds__(256, (PREC != PREC_F64 && NS <= 1) ? 4 : 1) k_stage(DevMesh mesh, StageArgs a)
{
    using R = typename PrecT<PREC>::R;
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = (int)(gt / LPC), l = (int)(gt % LPC);
    const bool valid = c < mesh.n_cells;
    constexpr int P = ((NV + LPC - 1) / LPC) * LPC;
    R res[P];
#pragma unroll
    for (int v = 0; v < P; ++v) res[v] = (R)0;
    if (valid) {
        int s0, s1;
        slot_range(mesh, c, s0, s1);
        const bool own_flag = a.flags && a.flags[c];
        GlobalSrc<DIM, NV, PREC> src{a, mesh};
#pragma unroll 2
        for (int s = s0 + l; s < s1; s += LPC) {
            R F[NV];
            slot_flux<DIM, NV, NS, PREC>(mesh, a, src, c, s, own_flag, F);
#pragma unroll
            for (int v = 0; v < NV; ++v) res[v] += F[v];
        }
    }
    constexpr int B = P / LPC;
    if constexpr (LPC > 1) group_reduce_scatter<P, LPC, R>(res, l);
    if (!valid) return;
    R iv, dummy0, dummy1, dummy2;
    ld4<R>(Geo<R>::cellk(mesh) + 4ll * c, dummy0, dummy1, dummy2, iv);
    const long long n = mesh.n_cells;
    bool bad = false;
    using T0 = typename PrecT<PREC>::T0;
    T0 *nxt = static_cast<T0 *>(a.o0_next);
    constexpr int S0 = ord_stride<DIM, NV, 0, PREC>();
    const R dtr = (R)a.dt;
#pragma unroll
    for (int i = 0; i < B; ++i) {
        const int v = l * B + i;
        if (v < NV) {
            const R r = res[i] * iv;
            if constexpr (PREC != PREC_F64) {
                if (a.mode == 2) {
                    bad |= incr_update<R, T0, S0>(a, c, v, n, r, dtr, nxt);
                    continue;
                }
            }
            double o;
            if (a.mode == 0) {
                o = (double)r;
                bad |= !isfinite(r);
            } else {
                o = stage_update(a, v * n + c, r * dtr);
                bad |= nonfinite64(o);
                if (nxt) nxt[c * (long long)S0 + v] = (T0)o;
            }
            a.out[v * n + c] = o;
        }
    }
    if (bad) atomicOr(a.status, 1u);
}

// Residual R_c = res / V_c and the stage output of one cell (one thread per cell):
// mode 0 the FP64 residual, mode 1 the FP64 stage value (+ next order-0 record),
// mode 2 the increment form.
template <int DIM, int NV, int PREC>
__device__ __forceinline__ void cell_epilogue(const DevMesh &mesh, const StageArgs &a, int c,
                                              const typename PrecT<PREC>::R *res)
{
    using R = typename PrecT<PREC>::R;
    R iv, dummy0, dummy1, dummy2;
    ld4<R>(Geo<R>::cellk(mesh) + 4ll * c, dummy0, dummy1, dummy2, iv);
    const long long n = mesh.n_cells;
    bool bad = false;
    using T0 = typename PrecT<PREC>::T0;
    T0 *nxt = static_cast<T0 *>(a.o0_next);
    constexpr int S0 = ord_stride<DIM, NV, 0, PREC>();
    R nv_out[NV];
    const R dtr = (R)a.dt;
    if constexpr (PREC != PREC_F64) {
        if (a.mode == 2) {
            R r[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) r[v] = res[v] * iv;
            bad = incr_update_cell<NV, R, T0, S0>(a, c, n, r, dtr, nxt);
            if (bad) atomicOr(a.status, 1u);
            return;
        }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const R r = res[v] * iv;
        const double o = a.mode == 0 ? (double)r : stage_update(a, v * n + c, r * dtr);
        nv_out[v] = (R)o;
        a.out[v * n + c] = o;
        bad |= nonfinite64(o);
    }
    if (a.mode != 0 && nxt) store_rec<T0, NV, S0, R>(nxt, c, nv_out);
    if (bad) atomicOr(a.status, 1u);
}

// ------------------------------------------------------------------ Dirichlet / Neumann faces
// After the first differential pass (which gives every boundary face the cell's own
// value): each cell with Dirichlet/Neumann faces adds S_f (T_f - T_C) / V_c per such
// face to its first-order record, so that the Gauss gradient takes the boundary face
// value T_f (Sec 2.6).  Higher orders keep the cell's own differentials on the face.
template <int DIM, int NV, int PREC>
__global__ void __launch_bounds__(128) k_bnd_grad(DevMesh mesh, const void *__restrict__ o0_v, void *__restrict__ o1_v)
{
    using R = typename PrecT<PREC>::R;
    using T0 = typename OrdT<PREC, 0>::T;
    using T1 = typename OrdT<PREC, 1>::T;
    constexpr int S0 = ord_stride<DIM, NV, 0, PREC>(), S1 = ord_stride<DIM, NV, 1, PREC>();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= mesh.n_bcell) return;
    const int c = __ldg(mesh.bcell + i);
    R U[NV], G[NV * DIM];
    load_rec<T0, NV, S0, R>(static_cast<const T0 *>(o0_v), c, U);
    T1 *o1 = static_cast<T1 *>(o1_v);
    load_rec<T1, NV * DIM, S1, R, false>(o1, c, G);
    R w0, w1, w2, iv;
    ld4<R>(Geo<R>::cellk(mesh) + 4ll * c, w0, w1, w2, iv);
    for (int k = __ldg(mesh.bcell_off + i); k < __ldg(mesh.bcell_off + i + 1); ++k) {
        const int f = __ldg(mesh.bcell_face + k);
        R fr[8];
        {
            const R *p = Geo<R>::face(mesh) + 8ll * f;
            ld4<R>(p, fr[0], fr[1], fr[2], fr[3]);
            ld4<R>(p + 4, fr[4], fr[5], fr[6], fr[7]);
        }
        R Uf[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) Uf[v] = U[v];
        boundary_state<NV, R>(mesh, f, Uf);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const R dT = (Uf[v] - U[v]) * iv;
            G[v * DIM + 0] += fr[4] * dT;
            G[v * DIM + 1] += fr[5] * dT;
            if constexpr (DIM == 3) G[v * DIM + 2] += fr[6] * dT;
        }
    }
    store_rec<T1, NV * DIM, S1, R>(o1, c, G);
}

// ------------------------------------------------------------------ face-centric pair
// k_flux evaluates every face once (thread per face, faces in owner order, canonical
// owner -> neighbour orientation, a boundary face the flux of its cell's state) into
// face_flux; k_gather then sums each cell's signed fluxes in slot order and applies
// the stage epilogue.  The operands and the order of the sums are those of the
// one-thread-per-cell kernel, whose results this pair reproduces.
template <int DIM, int NV, int NS, int PREC>
__global__ void __launch_bounds__(256) k_flux(DevMesh mesh, StageArgs a)
{
    using R = typename PrecT<PREC>::R;
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= mesh.n_faces) return;
    const int P = __ldg(mesh.fo + f), N = __ldg(mesh.fn + f);
    const unsigned word = ((unsigned)f << 2) | (N < 0 ? 2u : 0u);
    GlobalSrc<DIM, NV, PREC> src{a, mesh};
    const bool own_flag = a.flags && a.flags[P];
    R F[NV];
    canon_flux<DIM, NV, NS, PREC>(a, src, P, N < 0 ? P : N, word, own_flag, F);
    R *out = static_cast<R *>(a.face_flux);
    const long long nf = mesh.n_faces;
#pragma unroll
    for (int v = 0; v < NV; ++v) out[v * nf + f] = F[v];
}

template <int DIM, int NV, int PREC>
__global__ void __launch_bounds__(256) k_gather(DevMesh mesh, StageArgs a)
{
    using R = typename PrecT<PREC>::R;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= mesh.n_cells) return;
    const R *flux = static_cast<const R *>(a.face_flux);
    const long long nf = mesh.n_faces;
    R res[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) res[v] = (R)0;
    int s0, s1;
    slot_range(mesh, c, s0, s1);
    auto slot = [&](unsigned word) {
        const long long f = (long long)(word >> 2);
        const bool side = word & 1;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const R F = __ldg(flux + v * nf + f);
            res[v] += side ? F : -F;
        }
    };
    if (s1 - s0 == 4 && (s0 & 3) == 0) {
        // the four slot words of a four-slot cell (tetrahedron, quad): one aligned
        // 16-byte load
        const uint4 w = __ldg(reinterpret_cast<const uint4 *>(mesh.sword + s0));
        slot(w.x);
        slot(w.y);
        slot(w.z);
        slot(w.w);
    } else {
        for (int s = s0; s < s1; ++s) slot(__ldg(mesh.sword + s));
    }
    cell_epilogue<DIM, NV, PREC>(mesh, a, c, res);
}

// ------------------------------------------------------------------ tiled variants
// The block's TILE consecutive (Morton-ordered) cells stage their records, and the
// faces they own, in shared memory with asynchronous copies; neighbours inside the
// tile are then read from shared memory and only the tile's halo from global memory.
__device__ __forceinline__ void block_copy(unsigned char *dst, const unsigned char *src, unsigned bytes)
{
    const unsigned n16 = bytes / 16;
    for (unsigned i = threadIdx.x; i < n16; i += blockDim.x) {
        const unsigned sa = (unsigned)__cvta_generic_to_shared(dst + 16 * i);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(src + 16 * i));
    }
    for (unsigned i = 16 * n16 + 2 * threadIdx.x; i < bytes; i += 2 * blockDim.x)
        *reinterpret_cast<unsigned short *>(dst + i) = *reinterpret_cast<const unsigned short *>(src + i);
}
__device__ __forceinline__ void block_copy_wait()
{
    asm volatile("cp.async.commit_group;\n" ::);
    asm volatile("cp.async.wait_group 0;\n" ::);
    __syncthreads();
}

DOL_HD constexpr unsigned r16(unsigned b) { return (b + 15u) & ~15u; }

template <int DIM, int NV, int NS, int PREC, int TILE> struct TileLayout {
    template <int M> static DOL_HD constexpr unsigned bytes()
    {
        return r16((unsigned)TILE * ord_stride<DIM, NV, M, PREC>() * (unsigned)sizeof(typename OrdT<PREC, M>::T));
    }
    static DOL_HD constexpr unsigned off(int m)
    {
        return (m > 0 ? bytes<0>() : 0) + (m > 1 ? bytes<1>() : 0) + (m > 2 ? bytes<2>() : 0) + (m > 3 ? bytes<3>() : 0) +
               (m > 4 ? bytes<4>() : 0);
    }
};

template <int DIM, int NV, int NS, int PREC, int TILE>
__global__ void __launch_bounds__(TILE) k_stage_tile(DevMesh mesh, StageArgs a)
{
    using R = typename PrecT<PREC>::R;
    using L = TileLayout<DIM, NV, NS, PREC, TILE>;
    extern __shared__ __align__(16) unsigned char sm[];
    const int t0 = blockIdx.x * TILE;
    const int nt = min(TILE, mesh.n_cells - t0);
    TileSrc<DIM, NV, NS, PREC> src{a, mesh, sm, t0, nt, __ldg(mesh.fown + t0), __ldg(mesh.fown + t0 + nt), {}};
#pragma unroll
    for (int m = 0; m <= NS + 1; ++m) src.off[m] = L::off(m);
    auto copy_order = [&](auto mc) {
        constexpr int M = decltype(mc)::value;
        using T = typename OrdT<PREC, M>::T;
        constexpr unsigned rb = ord_stride<DIM, NV, M, PREC>() * (unsigned)sizeof(T);
        block_copy(sm + L::off(M), static_cast<const unsigned char *>(a.ord[M]) + (long long)t0 * rb, nt * rb);
    };
    copy_order(std::integral_constant<int, 0>{});
    if constexpr (NS >= 1) copy_order(std::integral_constant<int, 1>{});
    if constexpr (NS >= 2) copy_order(std::integral_constant<int, 2>{});
    if constexpr (NS >= 3) copy_order(std::integral_constant<int, 3>{});
    if constexpr (NS >= 4) copy_order(std::integral_constant<int, 4>{});
    block_copy(sm + L::off(NS + 1), reinterpret_cast<const unsigned char *>(Geo<R>::face(mesh) + 8ll * src.f_lo),
               (unsigned)(src.f_hi - src.f_lo) * 8u * (unsigned)sizeof(R));
    block_copy_wait();
    const int c = t0 + threadIdx.x;
    if (c >= mesh.n_cells) return;
    R res[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) res[v] = (R)0;
    int s0, s1;
    slot_range(mesh, c, s0, s1);
    const bool own_flag = a.flags && a.flags[c];
    for (int s = s0; s < s1; ++s) {
        R F[NV];
        slot_flux<DIM, NV, NS, PREC>(mesh, a, src, c, s, own_flag, F);
#pragma unroll
        for (int v = 0; v < NV; ++v) res[v] += F[v];
    }
    cell_epilogue<DIM, NV, PREC>(mesh, a, c, res);
}

template <int DIM, int NV, int M, int PREC, int TILE>
__global__ void __launch_bounds__(TILE) k_diff_tile(DevMesh mesh, const void *__restrict__ in_v, void *__restrict__ out_v)
{
    using R = typename PrecT<PREC>::R;
    using TI = typename OrdT<PREC, M - 1>::T;
    using TO = typename OrdT<PREC, M>::T;
    constexpr int CI = ncoef(DIM, M - 1), CO = ncoef(DIM, M);
    constexpr int SI = ord_stride<DIM, NV, M - 1, PREC>(), SO = ord_stride<DIM, NV, M, PREC>();
    extern __shared__ __align__(16) unsigned char sm[];
    const TI *in = static_cast<const TI *>(in_v);
    TO *out = static_cast<TO *>(out_v);
    const int t0 = blockIdx.x * TILE;
    const int nt = min(TILE, mesh.n_cells - t0);
    block_copy(sm, reinterpret_cast<const unsigned char *>(in + (long long)t0 * SI), (unsigned)nt * SI * sizeof(TI));
    block_copy_wait();
    const TI *tin = reinterpret_cast<const TI *>(sm);
    const int c = t0 + threadIdx.x;
    constexpr unsigned RBO = SO * (unsigned)sizeof(TO);
    const bool valid = c < mesh.n_cells;
    R acc[NV * CO];
#pragma unroll
    for (int i = 0; i < NV * CO; ++i) acc[i] = (R)0;
    if (valid) {
        R x[NV * CI];
        R wx, wy, wz, iv;
        ld4<R>(Geo<R>::cellk(mesh) + 4ll * c, wx, wy, wz, iv);
        load_rec<TI, NV * CI, SI, R, false>(tin, threadIdx.x, x);
        poly_mul_acc<DIM, NV, M, R>(acc, x, wx, wy, wz);
        int s0, s1;
        slot_range(mesh, c, s0, s1);
        constexpr int UB = diff_batch(NV * CI);
        for (int s = s0; s < s1; s += UB) {
            R kx[UB], ky[UB], kz[UB];
            int nbv[UB];
            bool ok[UB];
#pragma unroll
            for (int u = 0; u < UB; ++u) {
                ok[u] = s + u < s1;
                R kb = (R)0;
                kx[u] = ky[u] = kz[u] = (R)0;
                if (ok[u]) ld4<R>(Geo<R>::slotk(mesh) + 4ll * (s + u), kx[u], ky[u], kz[u], kb);
                nbv[u] = Geo<R>::nb_of(kb);
            }
            R xs[UB][NV * CI];
#pragma unroll
            for (int u = 0; u < UB; ++u) {
                if (!ok[u]) continue;
                const unsigned i = (unsigned)(nbv[u] - t0);
                if (i < (unsigned)nt) load_rec<TI, NV * CI, SI, R, false>(tin, i, xs[u]);
                else load_rec<TI, NV * CI, SI, R>(in, nbv[u], xs[u]);
            }
#pragma unroll
            for (int u = 0; u < UB; ++u)
                if (ok[u]) poly_mul_acc<DIM, NV, M, R>(acc, xs[u], kx[u], ky[u], kz[u]);
        }
    }
    if constexpr (RBO % 16 == 0) {
        // the tile's output records are contiguous: one bulk copy from shared memory
        unsigned char *so = sm + r16((unsigned)TILE * SI * (unsigned)sizeof(TI));
        if (valid) store_rec_smem<TO, NV * CO, SO, R>(so, threadIdx.x, acc);
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) bulk_s2g_wait(out + (long long)t0 * SO, so, (unsigned)nt * RBO);
    } else {
        if (valid) store_rec<TO, NV * CO, SO, R>(out, c, acc);
    }
}

// ------------------------------------------------------------------ persistent batched stage
// One cooperative launch runs a whole stage over the concatenated meshes of a batch:
// [pack the FP64 field] | differential pass 1 | ... | pass n_diff | reconstruction,
// flux, residual and update, the phases separated by a grid-wide barrier.  Records
// written in one phase are read in a later phase of the same launch, so this kernel
// reads through the coherent path (no read-only loads).  Each barrier waits at most
// `spin_limit` polls; a wait that gives up sets status bit 1 and an abort word that
// makes every later barrier of the launch return at once.
struct BatchArgs {
    const double *pack_src;      // non-null: phase 0 packs this FP64 field into ord[0]
    void *ord[MAXN + 1];         // order records 0..n_diff
    int n_diff;
    const int32_t *cell_mesh;    // mesh of each cell
    const double *dt_tab;        // per-mesh time step
    unsigned *bar;               // [0] arrivals, [32] generation, [64] abort
    unsigned spin_limit;
};

__device__ __forceinline__ void grid_barrier(unsigned *bar, unsigned *status, unsigned limit)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = bar + 32, *abort = bar + 64;
        if (!*abort) {
            const unsigned g = *gen;
            __threadfence();
            const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
            if (atomicAdd(bar, 1u) == nb - 1) {
                atomicExch(bar, 0u);
                __threadfence();
                atomicAdd(const_cast<unsigned *>(gen), 1u);
            } else {
                unsigned it = 0;
                while (*gen == g && !*abort) {
                    if (++it > limit) {
                        atomicOr(status, 2u);
                        atomicExch(const_cast<unsigned *>(abort), 1u);
                        break;
                    }
                    __nanosleep(100);
                }
            }
            __threadfence();
        }
    }
    __syncthreads();
}

template <int DIM, int NV, int M, int PREC>
__device__ __forceinline__ void diff_cell(const DevMesh &mesh, const void *in_v, void *out_v, int c)
{
    using R = typename PrecT<PREC>::R;
    using TI = typename OrdT<PREC, M - 1>::T;
    using TO = typename OrdT<PREC, M>::T;
    constexpr int CI = ncoef(DIM, M - 1), CO = ncoef(DIM, M);
    constexpr int SI = ord_stride<DIM, NV, M - 1, PREC>(), SO = ord_stride<DIM, NV, M, PREC>();
    const TI *in = static_cast<const TI *>(in_v);
    R acc[NV * CO];
#pragma unroll
    for (int i = 0; i < NV * CO; ++i) acc[i] = (R)0;
    R x[NV * CI];
    R wx, wy, wz, iv;
    ld4<R>(Geo<R>::cellk(mesh) + 4ll * c, wx, wy, wz, iv);
    load_rec<TI, NV * CI, SI, R, false>(in, c, x);
    poly_mul_acc<DIM, NV, M, R>(acc, x, wx, wy, wz);
    int s0, s1;
    slot_range(mesh, c, s0, s1);
    for (int s = s0; s < s1; ++s) {
        R kx, ky, kz, kb;
        ld4<R>(Geo<R>::slotk(mesh) + 4ll * s, kx, ky, kz, kb);
        load_rec<TI, NV * CI, SI, R, false>(in, Geo<R>::nb_of(kb), x);
        poly_mul_acc<DIM, NV, M, R>(acc, x, kx, ky, kz);
    }
    store_rec<TO, NV * CO, SO, R>(static_cast<TO *>(out_v), c, acc);
}

template <int DIM, int NV, int PREC> struct CoherentSrc {
    using R = typename PrecT<PREC>::R;
    static constexpr bool LDG = false;
    const StageArgs &a;
    const DevMesh &mesh;
    template <int M> __device__ __forceinline__ const typename OrdT<PREC, M>::T *rec(int X) const
    {
        return static_cast<const typename OrdT<PREC, M>::T *>(a.ord[M]) + (long long)X * ord_stride<DIM, NV, M, PREC>();
    }
    __device__ __forceinline__ const R *face(int f) const { return Geo<R>::face(mesh) + 8ll * f; }
};

template <int DIM, int NV, int NS, int PREC>
__global__ void __launch_bounds__(256) k_batch_stage(DevMesh mesh, StageArgs a, BatchArgs b)
{
    using R = typename PrecT<PREC>::R;
    using T0 = typename PrecT<PREC>::T0;
    const int nthr = gridDim.x * blockDim.x;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = mesh.n_cells;
    constexpr int S0 = ord_stride<DIM, NV, 0, PREC>();
    if (b.pack_src) {
        for (int c = tid; c < n; c += nthr) {
            R v[NV];
#pragma unroll
            for (int i = 0; i < NV; ++i) v[i] = (R)b.pack_src[(long long)i * n + c];
            store_rec<T0, NV, S0, R>(static_cast<T0 *>(b.ord[0]), c, v);
        }
        grid_barrier(b.bar, a.status, b.spin_limit);
    }
    if (b.n_diff >= 1) {
        for (int c = tid; c < n; c += nthr) diff_cell<DIM, NV, 1, PREC>(mesh, b.ord[0], b.ord[1], c);
        grid_barrier(b.bar, a.status, b.spin_limit);
    }
    if (b.n_diff >= 2) {
        for (int c = tid; c < n; c += nthr) diff_cell<DIM, NV, 2, PREC>(mesh, b.ord[1], b.ord[2], c);
        grid_barrier(b.bar, a.status, b.spin_limit);
    }
    if (b.n_diff >= 3) {
        for (int c = tid; c < n; c += nthr) diff_cell<DIM, NV, 3, PREC>(mesh, b.ord[2], b.ord[3], c);
        grid_barrier(b.bar, a.status, b.spin_limit);
    }
    if (b.n_diff >= 4) {
        for (int c = tid; c < n; c += nthr) diff_cell<DIM, NV, 4, PREC>(mesh, b.ord[3], b.ord[4], c);
        grid_barrier(b.bar, a.status, b.spin_limit);
    }
    if (*(volatile unsigned *)(b.bar + 64)) return;      // a barrier gave up: leave the state untouched
    CoherentSrc<DIM, NV, PREC> src{a, mesh};
    T0 *nxt = static_cast<T0 *>(a.o0_next);
    for (int c = tid; c < n; c += nthr) {
        R res[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) res[v] = (R)0;
        int s0, s1;
        slot_range(mesh, c, s0, s1);
        const bool own_flag = a.flags && a.flags[c];
        for (int s = s0; s < s1; ++s) {
            R F[NV];
            slot_flux<DIM, NV, NS, PREC>(mesh, a, src, c, s, own_flag, F);
#pragma unroll
            for (int v = 0; v < NV; ++v) res[v] += F[v];
        }
        R iv, d0, d1, d2;
        ld4<R>(Geo<R>::cellk(mesh) + 4ll * c, d0, d1, d2, iv);
        const R dtr = (R)b.dt_tab[__ldg(b.cell_mesh + c)];
        bool bad = false;
        R o32[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const R r = res[v] * iv;
            const double o = stage_update(a, (long long)v * n + c, r * dtr);
            a.out[(long long)v * n + c] = o;
            o32[v] = (R)o;
            bad |= nonfinite64(o);
        }
        if (nxt) store_rec<T0, NV, S0, R>(nxt, c, o32);
        if (bad) atomicOr(a.status, 1u);
    }
}

// ------------------------------------------------------------------ face states (diagnostic)
template <int DIM, int NV, int NS, int PREC>
__global__ void __launch_bounds__(128) k_faces(DevMesh mesh, StageArgs a, double *fL, double *fR)
{
    using R = typename PrecT<PREC>::R;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= mesh.n_faces) return;
    const int P = mesh.fo[i], N = mesh.fn[i];
    const long long e = mesh.face_ext[i];
    const bool flip = mesh.face_flip[i];
    R fr[8];
    {
        const R *p = Geo<R>::face(mesh) + 8ll * i;
        ld4<R>(p, fr[0], fr[1], fr[2], fr[3]);
        ld4<R>(p + 4, fr[4], fr[5], fr[6], fr[7]);
    }
    R UL[NV], UR[NV];
    if (N < 0) {
        load_rec<typename PrecT<PREC>::T0, NV, ord_stride<DIM, NV, 0, PREC>(), R>(
            static_cast<const typename PrecT<PREC>::T0 *>(a.ord[0]), P, UL);
        boundary_state<NV, R>(mesh, i, UL);
#pragma unroll
        for (int v = 0; v < NV; ++v) UR[v] = UL[v];
    } else {
        const int lim = face_limit(a, a.flags && (a.flags[P] || a.flags[N]));
        GlobalSrc<DIM, NV, PREC> src{a, mesh};
        face_states<DIM, NV, NS, PREC, false>(a, src, fr, i, P, N, lim, UL, UR, true);
    }
    const long long nf = mesh.n_faces;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        fL[v * nf + e] = (double)(flip ? UR[v] : UL[v]);
        fR[v * nf + e] = (double)(flip ? UL[v] : UR[v]);
    }
}

}  // namespace dol
