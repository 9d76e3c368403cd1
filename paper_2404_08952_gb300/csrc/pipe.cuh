// Persistent, pipelined gather kernels for sm_103a.
//
// A CTA walks over tiles of consecutive (Morton-ordered) cells.  For each tile one
// elected thread issues bulk asynchronous copies (cp.async.bulk, the TMA 1D form)
// of the tile's contiguous arrays -- its input records, per-cell and per-slot
// geometry -- into one of two shared-memory buffers, completing on an mbarrier;
// while the CTA computes tile j from one buffer, tile j+1 is already in flight into
// the other.  Neighbours inside the tile are read from shared memory, the tile's
// halo from global memory.  The arithmetic and its order are those of the
// non-pipelined kernels, so results are bit-identical for the same lanes per cell.
//
// Every mbarrier wait is bounded; a wait that gives up sets status bit 1 (reported
// as DOLINC_ERR_DEVICE_TIMEOUT).  Then, before the CTA leaves (without writing the
// tile), every thread waits again for each bulk copy the CTA has in flight -- the
// current tile's and the next tile's, both issued by thread 0 before its wait -- with
// a longer bound (kPipeDrainLimit), so that no copy lands in the shared memory of a
// CTA that has exited.  Only a GPU that stopped completing copies altogether gets
// past both bounds; the kernel then returns rather than hang.
#pragma once
#include "kernels.cuh"

namespace dol {

constexpr unsigned kPipeWaitLimit = 1u << 22;   // try_wait polls before a wait gives up
constexpr unsigned kPipeDrainLimit = 1u << 25;  // polls per in-flight copy on the give-up path

DOL_HD constexpr unsigned al128(unsigned b) { return (b + 127u) & ~127u; }

// ------------------------------------------------------------------ differential pass
// Shared-memory buffer of one tile: input records, cell geometry, slot geometry.
template <int DIM, int NV, int M, int PREC, int TC> struct DiffPipeLayout {
    using R = typename PrecT<PREC>::R;
    using TI = typename OrdT<PREC, M - 1>::T;
    static constexpr unsigned RB = ord_stride<DIM, NV, M - 1, PREC>() * (unsigned)sizeof(TI);
    static constexpr unsigned rec_bytes = al128(TC * RB);
    static constexpr unsigned cell_bytes = al128(TC * 4u * (unsigned)sizeof(R));
    static DOL_HD unsigned slot_bytes(int max_faces) { return al128((unsigned)(TC * max_faces) * 4u * (unsigned)sizeof(R)); }
    static DOL_HD unsigned buf_bytes(int max_faces) { return rec_bytes + cell_bytes + slot_bytes(max_faces); }
    static DOL_HD unsigned smem_bytes(int max_faces) { return 128u + 2u * buf_bytes(max_faces); }
};

template <int DIM, int NV, int M, int PREC, int LPC, int NT>
__global__ void __launch_bounds__(NT) k_diff_pipe(DevMesh mesh, const void *__restrict__ in_v, void *__restrict__ out_v,
                                                 unsigned *status, int max_faces)
{
    using R = typename PrecT<PREC>::R;
    using TI = typename OrdT<PREC, M - 1>::T;
    using TO = typename OrdT<PREC, M>::T;
    constexpr int TC = NT / LPC;
    using L = DiffPipeLayout<DIM, NV, M, PREC, TC>;
    constexpr int CI = ncoef(DIM, M - 1), CO = ncoef(DIM, M);
    constexpr int SI = ord_stride<DIM, NV, M - 1, PREC>(), SO = ord_stride<DIM, NV, M, PREC>();
    const TI *in = static_cast<const TI *>(in_v);
    TO *out = static_cast<TO *>(out_v);
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm);
    const unsigned bb = L::buf_bytes(max_faces);
    const int n_tiles = (mesh.n_cells + TC - 1) / TC;
    if ((int)blockIdx.x >= n_tiles) return;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        mbar_fence_init();
    }
    __syncthreads();

    // producer: tile -> buffer b
    auto issue = [&](int tile, int b) {
        const int t0 = tile * TC, nt = min(TC, mesh.n_cells - t0);
        unsigned char *buf = sm + 128 + b * bb;
        const unsigned rb = ((unsigned)nt * L::RB) & ~15u;
        const unsigned cb = (unsigned)nt * 4u * (unsigned)sizeof(R);
        const int s_lo = __ldg(mesh.off + t0), s_hi = __ldg(mesh.off + t0 + nt);
        const unsigned sb = (unsigned)(s_hi - s_lo) * 4u * (unsigned)sizeof(R);
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar + b, rb + cb + sb);
        if (rb) bulk_g2s(buf, reinterpret_cast<const unsigned char *>(in) + (long long)t0 * L::RB, rb, bar + b);
        bulk_g2s(buf + L::rec_bytes, Geo<R>::cellk(mesh) + 4ll * t0, cb, bar + b);
        if (sb) bulk_g2s(buf + L::rec_bytes + L::cell_bytes, Geo<R>::slotk(mesh) + 4ll * s_lo, sb, bar + b);
    };

    if (threadIdx.x == 0) issue(blockIdx.x, 0);
    const int l = threadIdx.x % LPC, ci = threadIdx.x / LPC;
    for (int j = 0, tile = blockIdx.x; tile < n_tiles; ++j, tile += gridDim.x) {
        const int b = j & 1;
        const int next = tile + gridDim.x;
        if (threadIdx.x == 0 && next < n_tiles) issue(next, b ^ 1);
        const bool ok = mbar_wait(bar + b, (unsigned)(j >> 1) & 1u, kPipeWaitLimit);
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) atomicOr(status, 2u);
            if (!ok) mbar_wait(bar + b, (unsigned)(j >> 1) & 1u, kPipeDrainLimit);
            if (next < n_tiles) mbar_wait(bar + (b ^ 1), (unsigned)((j + 1) >> 1) & 1u, kPipeDrainLimit);
            return;
        }
        const unsigned char *buf = sm + 128 + b * bb;
        const TI *trec = reinterpret_cast<const TI *>(buf);
        const R *tcell = reinterpret_cast<const R *>(buf + L::rec_bytes);
        const R *tslot = reinterpret_cast<const R *>(buf + L::rec_bytes + L::cell_bytes);
        const int t0 = tile * TC, nt = min(TC, mesh.n_cells - t0);
        const int n_staged = (int)((((unsigned)nt * L::RB) & ~15u) / L::RB);   // records fully in the buffer
        const int c = t0 + ci;
        const bool valid = ci < nt;
        constexpr int VO = 16 / (int)sizeof(TO);
        constexpr int P = (LPC == 1) ? NV * CO : round_up(SO, LPC * VO);
        R acc[P];
#pragma unroll
        for (int i = 0; i < P; ++i) acc[i] = (R)0;
        if (valid) {
            R x[NV * CI];
            const int s_base = __ldg(mesh.off + t0);
            if (l == 0) {
                R wx, wy, wz, iv;
                ld4<R, false>(tcell + 4 * ci, wx, wy, wz, iv);
                if (ci < n_staged) load_rec<TI, NV * CI, SI, R, false>(trec, ci, x);
                else load_rec<TI, NV * CI, SI, R>(in, c, x);
                poly_mul_acc<DIM, NV, M, R>(acc, x, wx, wy, wz);
            }
            int s0, s1;
            slot_range(mesh, c, s0, s1);
            for (int s = s0 + l; s < s1; s += LPC) {
                R kx, ky, kz, kb;
                ld4<R, false>(tslot + 4 * (s - s_base), kx, ky, kz, kb);
                const int nb = Geo<R>::nb_of(kb);
                const unsigned i = (unsigned)(nb - t0);
                if (i < (unsigned)n_staged) load_rec<TI, NV * CI, SI, R, false>(trec, i, x);
                else load_rec<TI, NV * CI, SI, R>(in, nb, x);
                poly_mul_acc<DIM, NV, M, R>(acc, x, kx, ky, kz);
            }
        }
        if constexpr (LPC == 1) {
            if (valid) store_rec<TO, NV * CO, SO, R>(out, c, acc);
        } else {
            group_reduce_scatter<P, LPC, R>(acc, l);
            if (valid) {
                constexpr int B = P / LPC;
                const int e0 = l * B;
                TO *rec = out + (long long)c * SO;
#pragma unroll
                for (int i = 0; i < B; ++i)
                    if (e0 + i < NV * CO) rec[e0 + i] = to_store<TO, R>(acc[i]);
            }
        }
        __syncthreads();   // buffer b is free for tile j+2
    }
}

// ------------------------------------------------------------------ fused stage
// Tile-local face-centric stage.  Phase A evaluates each face the tile needs once:
// the faces its cells own (flux kept per face) and the faces whose owner lies in an
// earlier tile or outside the mesh (boundary slots; flux kept per slot); a face
// between two tiles is thus evaluated by both tiles, with identical operands in the
// canonical orientation, so the two results are bit-identical.  Phase B sums each
// cell's signed fluxes in slot order (the order of the one-thread-per-cell kernel,
// hence bit-identical results) and applies the stage epilogue.
template <int DIM, int NV, int NS, int PREC, int TC> struct StagePipeLayout {
    using R = typename PrecT<PREC>::R;
    template <int M> static DOL_HD constexpr unsigned RB()
    {
        return ord_stride<DIM, NV, M, PREC>() * (unsigned)sizeof(typename OrdT<PREC, M>::T);
    }
    // record bytes of order m (m = 0..4)
    static DOL_HD constexpr unsigned RBm(int m)
    {
        return m == 0 ? RB<0>() : m == 1 ? RB<1>() : m == 2 ? RB<2>() : m == 3 ? RB<3>() : RB<4>();
    }
    static DOL_HD constexpr unsigned rec_bytes(int m) { return al128(TC * RBm(m)); }
    static DOL_HD constexpr unsigned roff(int m)
    {
        unsigned o = 0;
        for (int i = 0; i < m; ++i) o += rec_bytes(i);
        return o;
    }
    static DOL_HD unsigned soff() { return roff(NS + 1); }
    static DOL_HD unsigned slot_bytes(int max_slots) { return al128((unsigned)(TC * max_slots + 2) * 8u); }
    static DOL_HD unsigned foff(int max_slots) { return soff() + slot_bytes(max_slots); }
    static DOL_HD unsigned face_bytes(int max_tf) { return al128((unsigned)max_tf * 8u * (unsigned)sizeof(R)); }
    static DOL_HD unsigned buf_bytes(int max_slots, int max_tf) { return foff(max_slots) + face_bytes(max_tf); }
    static DOL_HD unsigned fbuf_bytes(int max_tf) { return al128((unsigned)max_tf * NV * (unsigned)sizeof(R)); }
    static DOL_HD unsigned xbuf_bytes(int max_slots) { return al128((unsigned)(TC * max_slots) * NV * (unsigned)sizeof(R)); }
    static DOL_HD unsigned smem_bytes(int max_slots, int max_tf)
    {
        return 128u + 2u * buf_bytes(max_slots, max_tf) + fbuf_bytes(max_tf) + xbuf_bytes(max_slots);
    }
};

template <int DIM, int NV, int NS, int PREC, int TC, int NT>
__global__ void __launch_bounds__(NT) k_stage_pipe(DevMesh mesh, StageArgs a, int max_tf)
{
    using R = typename PrecT<PREC>::R;
    using L = StagePipeLayout<DIM, NV, NS, PREC, TC>;
    static_assert(NT % TC == 0, "threads per CTA must be a multiple of the tile");
    constexpr int LN = NT / TC;                  // phase-A lanes per cell
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm);
    const int max_slots = mesh.max_slots;
    const unsigned bb = L::buf_bytes(max_slots, max_tf);
    R *fbuf = reinterpret_cast<R *>(sm + 128 + 2 * bb);
    R *xbuf = reinterpret_cast<R *>(sm + 128 + 2 * bb + L::fbuf_bytes(max_tf));
    const int n_tiles = (mesh.n_cells + TC - 1) / TC;
    if ((int)blockIdx.x >= n_tiles) return;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        mbar_fence_init();
    }
    __syncthreads();

    auto issue = [&](int tile, int b) {
        const int t0 = tile * TC, nt = min(TC, mesh.n_cells - t0);
        unsigned char *buf = sm + 128 + b * bb;
        const int s_lo = __ldg(mesh.off + t0), s_hi = __ldg(mesh.off + t0 + nt);
        const int a_lo = s_lo & ~1;
        const unsigned sb = ((unsigned)(s_hi - a_lo) * 8u + 15u) & ~15u;
        const int f_lo = __ldg(mesh.fown + t0), f_hi = __ldg(mesh.fown + t0 + nt);
        const unsigned fb = (unsigned)(f_hi - f_lo) * 8u * (unsigned)sizeof(R);
        unsigned rb[NS + 1];
        unsigned tx = sb + fb;
#pragma unroll
        for (int m = 0; m <= NS; ++m) {
            const unsigned rbm = L::RBm(m);
            rb[m] = ((unsigned)nt * rbm) & ~15u;
            tx += rb[m];
        }
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar + b, tx);
#pragma unroll
        for (int m = 0; m <= NS; ++m) {
            const unsigned rbm = L::RBm(m);
            if (rb[m])
                bulk_g2s(buf + L::roff(m), static_cast<const unsigned char *>(a.ord[m]) + (long long)t0 * rbm, rb[m],
                         bar + b);
        }
        if (sb) bulk_g2s(buf + L::soff(), mesh.slot2 + a_lo, sb, bar + b);
        if (fb) bulk_g2s(buf + L::foff(max_slots), Geo<R>::face(mesh) + 8ll * f_lo, fb, bar + b);
    };

    if (threadIdx.x == 0) issue(blockIdx.x, 0);
    for (int j = 0, tile = blockIdx.x; tile < n_tiles; ++j, tile += gridDim.x) {
        const int b = j & 1;
        const int next = tile + gridDim.x;
        if (threadIdx.x == 0 && next < n_tiles) issue(next, b ^ 1);
        const bool ok = mbar_wait(bar + b, (unsigned)(j >> 1) & 1u, kPipeWaitLimit);
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) atomicOr(a.status, 2u);
            if (!ok) mbar_wait(bar + b, (unsigned)(j >> 1) & 1u, kPipeDrainLimit);
            if (next < n_tiles) mbar_wait(bar + (b ^ 1), (unsigned)((j + 1) >> 1) & 1u, kPipeDrainLimit);
            return;
        }
        const unsigned char *buf = sm + 128 + b * bb;
        const int t0 = tile * TC, nt = min(TC, mesh.n_cells - t0);
        const int s_lo = __ldg(mesh.off + t0);
        const int a_lo = s_lo & ~1;
        const int f_lo = __ldg(mesh.fown + t0), f_hi = __ldg(mesh.fown + t0 + nt);
        // records of cells [t0, t0 + n_staged) are in the buffer for every order
        int n_staged = nt;
#pragma unroll
        for (int m = 0; m <= NS; ++m) {
            const unsigned rbm = L::RBm(m);
            n_staged = min(n_staged, (int)((((unsigned)nt * rbm) & ~15u) / rbm));
        }
        TileSrc<DIM, NV, NS, PREC> src{a, mesh, buf, t0, n_staged, f_lo, f_hi, {}};
#pragma unroll
        for (int m = 0; m <= NS; ++m) src.off[m] = L::roff(m);
        src.off[NS + 1] = L::foff(max_slots);
        const int2 *ts = reinterpret_cast<const int2 *>(buf + L::soff());
        // phase A: the faces this tile evaluates
        {
            const int ci = threadIdx.x / LN, l = threadIdx.x % LN;
            if (ci < nt) {
                const int c = t0 + ci;
                int s0, s1;
                slot_range(mesh, c, s0, s1);
                const bool own_flag = a.flags && a.flags[c];
                for (int s = s0 + l; s < s1; s += LN) {
                    const int2 sw = ts[s - a_lo];
                    const unsigned word = (unsigned)sw.y;
                    const bool bnd = word & 2u, side = word & 1u;
                    const bool incoming = side && (unsigned)(sw.x - t0) >= (unsigned)nt;
                    if (side && !incoming) continue;        // the owner, in this tile, evaluates it
                    R F[NV];
                    canon_flux<DIM, NV, NS, PREC>(a, src, c, sw.x, word, own_flag, F);
                    R *dst = (bnd || incoming) ? xbuf + (long long)(s - s_lo) * NV
                                               : fbuf + (long long)((int)(word >> 2) - f_lo) * NV;
#pragma unroll
                    for (int v = 0; v < NV; ++v) dst[v] = F[v];
                }
            }
        }
        __syncthreads();
        // phase B: each cell sums its signed fluxes in slot order
        if ((int)threadIdx.x < nt) {
            const int c = t0 + threadIdx.x;
            int s0, s1;
            slot_range(mesh, c, s0, s1);
            R res[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) res[v] = (R)0;
            for (int s = s0; s < s1; ++s) {
                const int2 sw = ts[s - a_lo];
                const unsigned word = (unsigned)sw.y;
                const bool side = word & 1u;
                const bool per_slot = (word & 2u) || (side && (unsigned)(sw.x - t0) >= (unsigned)nt);
                const R *F = per_slot ? xbuf + (long long)(s - s_lo) * NV : fbuf + (long long)((int)(word >> 2) - f_lo) * NV;
#pragma unroll
                for (int v = 0; v < NV; ++v) res[v] += side ? F[v] : -F[v];
            }
            cell_epilogue<DIM, NV, PREC>(mesh, a, c, res);
        }
        (void)f_hi;
        __syncthreads();   // buffer b and the flux area are free
    }
}

}  // namespace dol
