// Host launchers of the templated stage kernels and the table the C ABI dispatches on.
#pragma once
#include <map>
#include <mutex>
#include "pipe.cuh"

namespace dol {

// Launch shape of the gather kernels: lanes per cell (1, 4 or 8; 0 = one thread per
// cell with the block's cells staged in shared memory, tile = block; -1 / -4 = the
// persistent pipelined kernel with 1 / 4 lanes per cell, block threads per CTA) and
// block size.
struct Tune {
    int diff_lpc = 4, diff_block = 256, stage_lpc = 4, stage_block = 128;
};

// Grid of a persistent kernel: resident CTAs per SM x SMs (cached per kernel and
// shared-memory size on the current device).
inline int persistent_grid(const void *kernel, int threads, size_t smem)
{
    static std::mutex mu;
    static std::map<std::tuple<int, const void *, size_t>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> g(mu);
    auto key = std::make_tuple(dev, kernel, smem);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
    const int grid = std::max(1, sms * std::max(per, 1));
    cache[key] = grid;
    return grid;
}

struct PathFns {
    void (*pack)(const DevMesh &, const double *, void *, double *copy, cudaStream_t);
    void (*diff)(const DevMesh &, int M, const void *, void *, const Tune &, unsigned *, cudaStream_t);
    // order 2 (inA -> outA) and order 1 (inB -> outB) in one launch; false (nothing
    // launched) where the records do not allow it; dry: only answer whether they do
    bool (*diff_pair)(const DevMesh &, const void *, void *, const void *, void *, cudaStream_t, bool dry);
    void (*stage)(const DevMesh &, const StageArgs &, const Tune &, cudaStream_t);
    void (*faces)(const DevMesh &, const StageArgs &, double *, double *, cudaStream_t);
    void (*bnd_grad)(const DevMesh &, const void *, void *, cudaStream_t);
};

inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }
constexpr size_t kMaxSmem = 200 * 1024;   // dynamic shared memory a tiled block may use

template <int DIM, int NV, int NS, int PREC> struct Path {
    static void pack(const DevMesh &m, const double *u, void *o0, double *copy, cudaStream_t s)
    {
        k_pack<NV, PREC><<<nblk(m.n_cells, 256), 256, 0, s>>>(m.n_cells, u,
                                                              static_cast<typename PrecT<PREC>::T0 *>(o0), copy);
    }
    // bytes of one output record of order MM, and the shared memory a block of bs
    // threads (one cell each) needs to stage its output records for the bulk store
    template <int MM> static constexpr unsigned out_rec_bytes()
    {
        return ord_stride<DIM, NV, MM, PREC>() * (unsigned)sizeof(typename OrdT<PREC, MM>::T);
    }
    template <int MM> static size_t out_smem(int bs)
    {
        return out_rec_bytes<MM>() % 16 == 0 ? (size_t)bs * out_rec_bytes<MM>() : 0;
    }
    // one thread per cell (lanes 1), output staged for the bulk store
    template <int MM> static void diff_1(const DevMesh &m, const void *in, void *out, int bs, cudaStream_t s)
    {
        static bool attr = false;   // opt in to more than 48 KB once per instantiation
        if (!attr) {
            cudaFuncSetAttribute(k_diff<DIM, NV, MM, PREC, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kMaxSmem);
            attr = true;
        }
        k_diff<DIM, NV, MM, PREC, 1><<<nblk(m.n_cells, bs), bs, out_smem<MM>(bs), s>>>(m, in, out);
    }
    template <int LPC> static void diff_l(const DevMesh &m, int M, const void *in, void *out, int bs, cudaStream_t s)
    {
        const int b = nblk((long long)m.n_cells * LPC, bs);
        if constexpr (LPC == 1) {
            switch (M) {
            case 1: diff_1<1>(m, in, out, bs, s); break;
            case 2: diff_1<2>(m, in, out, bs, s); break;
            case 3: diff_1<3>(m, in, out, bs, s); break;
            case 4: diff_1<4>(m, in, out, bs, s); break;
            default: break;
            }
            return;
        }
        switch (M) {
        case 1: k_diff<DIM, NV, 1, PREC, LPC><<<b, bs, 0, s>>>(m, in, out); break;
        case 2: k_diff<DIM, NV, 2, PREC, LPC><<<b, bs, 0, s>>>(m, in, out); break;
        case 3: k_diff<DIM, NV, 3, PREC, LPC><<<b, bs, 0, s>>>(m, in, out); break;
        case 4: k_diff<DIM, NV, 4, PREC, LPC><<<b, bs, 0, s>>>(m, in, out); break;
        default: break;
        }
    }
    template <int TILE> static void diff_t(const DevMesh &m, int M, const void *in, void *out, cudaStream_t s)
    {
        const int b = nblk(m.n_cells, TILE);
        auto sm = [&](auto mc) {
            constexpr int MM = decltype(mc)::value;
            const size_t in_b = (size_t)TILE * ord_stride<DIM, NV, MM - 1, PREC>() * sizeof(typename OrdT<PREC, MM - 1>::T);
            return ((in_b + 15) & ~(size_t)15) + out_smem<MM>(TILE);
        };
        auto go = [&](auto mc) {
            constexpr int MM = decltype(mc)::value;
            const size_t bytes = sm(mc);
            if (bytes > kMaxSmem) {                 // too large to stage: one thread per cell instead
                diff_1<MM>(m, in, out, TILE, s);
                return;
            }
            static bool attr = false;
            if (!attr) {
                cudaFuncSetAttribute(k_diff_tile<DIM, NV, MM, PREC, TILE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kMaxSmem);
                attr = true;
            }
            k_diff_tile<DIM, NV, MM, PREC, TILE><<<b, TILE, bytes, s>>>(m, in, out);
        };
        switch (M) {
        case 1: go(std::integral_constant<int, 1>{}); break;
        case 2: go(std::integral_constant<int, 2>{}); break;
        case 3: go(std::integral_constant<int, 3>{}); break;
        case 4: go(std::integral_constant<int, 4>{}); break;
        default: break;
        }
    }
    template <int TILE> static void stage_t(const DevMesh &m, const StageArgs &a, cudaStream_t s)
    {
        using L = TileLayout<DIM, NV, NS, PREC, TILE>;
        const int ti = TILE == 64 ? 0 : (TILE == 128 ? 1 : 2);
        const size_t sm = L::off(NS + 1) + (size_t)m.max_tile_faces[ti] * 8 * sizeof(typename PrecT<PREC>::R);
        if (sm > kMaxSmem) {                        // too large to stage: one thread per cell instead
            k_stage<DIM, NV, NS, PREC, 1><<<nblk(m.n_cells, TILE), TILE, 0, s>>>(m, a);
            return;
        }
        static bool attr = false;   // opt in to more than 48 KB once per instantiation
        if (!attr) {
            cudaFuncSetAttribute(k_stage_tile<DIM, NV, NS, PREC, TILE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kMaxSmem);
            attr = true;
        }
        k_stage_tile<DIM, NV, NS, PREC, TILE><<<nblk(m.n_cells, TILE), TILE, sm, s>>>(m, a);
    }
    template <int LPC, int NT>
    static void diff_p(const DevMesh &m, int M, const void *in, void *out, unsigned *status, cudaStream_t s)
    {
        auto go = [&](auto mc) {
            constexpr int MM = decltype(mc)::value;
            using L = DiffPipeLayout<DIM, NV, MM, PREC, NT / LPC>;
            const size_t bytes = L::smem_bytes(m.max_slots);
            if (bytes > kMaxSmem) {                 // too large to stage: one thread per cell instead
                diff_1<MM>(m, in, out, NT, s);
                return;
            }
            auto kern = k_diff_pipe<DIM, NV, MM, PREC, LPC, NT>;
            static bool attr = false;
            if (!attr) {
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
                attr = true;
            }
            const int tiles = nblk(m.n_cells, NT / LPC);
            const int grid = std::min(tiles, persistent_grid((const void *)kern, NT, bytes));
            kern<<<grid, NT, bytes, s>>>(m, in, out, status, m.max_slots);
        };
        switch (M) {
        case 1: go(std::integral_constant<int, 1>{}); break;
        case 2: go(std::integral_constant<int, 2>{}); break;
        case 3: go(std::integral_constant<int, 3>{}); break;
        case 4: go(std::integral_constant<int, 4>{}); break;
        default: break;
        }
    }
    static void diff(const DevMesh &m, int M, const void *in, void *out, const Tune &t, unsigned *status,
                     cudaStream_t s)
    {
        if (t.diff_lpc < 0) {
            const bool big = t.diff_block >= 256;
            if (t.diff_lpc == -4) big ? diff_p<4, 256>(m, M, in, out, status, s) : diff_p<4, 128>(m, M, in, out, status, s);
            else big ? diff_p<1, 256>(m, M, in, out, status, s) : diff_p<1, 128>(m, M, in, out, status, s);
            return;
        }
        if (t.diff_lpc == 0) {
            switch (t.diff_block) {
            case 64: diff_t<64>(m, M, in, out, s); break;
            case 256: diff_t<256>(m, M, in, out, s); break;
            default: diff_t<128>(m, M, in, out, s); break;
            }
            return;
        }
        switch (t.diff_lpc) {
        case 4: diff_l<4>(m, M, in, out, t.diff_block, s); break;
        case 8: diff_l<8>(m, M, in, out, t.diff_block, s); break;
        default: diff_l<1>(m, M, in, out, t.diff_block, s); break;
        }
    }
    template <int TC> static void stage_p(const DevMesh &m, const StageArgs &a, cudaStream_t s)
    {
        constexpr int NT = 256;
        using L = StagePipeLayout<DIM, NV, NS, PREC, TC>;
        const int max_tf = m.max_tile_faces[TC == 64 ? 0 : 1];
        const size_t bytes = L::smem_bytes(m.max_slots, max_tf);
        if (bytes > kMaxSmem) {                     // too large to stage: one thread per cell instead
            k_stage<DIM, NV, NS, PREC, 1><<<nblk(m.n_cells, 128), 128, 0, s>>>(m, a);
            return;
        }
        auto kern = k_stage_pipe<DIM, NV, NS, PREC, TC, NT>;
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
            attr = true;
        }
        const int grid = std::min(nblk(m.n_cells, TC), persistent_grid((const void *)kern, NT, bytes));
        kern<<<grid, NT, bytes, s>>>(m, a, max_tf);
    }
    static void stage(const DevMesh &m, const StageArgs &a, const Tune &t, cudaStream_t s)
    {
        if (t.stage_lpc == -2) {                    // face-centric pair
            k_flux<DIM, NV, NS, PREC><<<nblk(m.n_faces, 128), 128, 0, s>>>(m, a);
            k_gather<DIM, NV, PREC><<<nblk(m.n_cells, t.stage_block), t.stage_block, 0, s>>>(m, a);
            return;
        }
        if (t.stage_lpc < 0) {
            if (t.stage_block >= 128) stage_p<128>(m, a, s);
            else stage_p<64>(m, a, s);
            return;
        }
        if (t.stage_lpc == 0) {
            switch (t.stage_block) {
            case 64: stage_t<64>(m, a, s); break;
            case 256: stage_t<256>(m, a, s); break;
            default: stage_t<128>(m, a, s); break;
            }
            return;
        }
        const int bs = t.stage_block;
        switch (t.stage_lpc) {
        case 4: k_stage<DIM, NV, NS, PREC, 4><<<nblk((long long)m.n_cells * 4, bs), bs, 0, s>>>(m, a); break;
        case 8: k_stage<DIM, NV, NS, PREC, 8><<<nblk((long long)m.n_cells * 8, bs), bs, 0, s>>>(m, a); break;
        default: k_stage<DIM, NV, NS, PREC, 1><<<nblk(m.n_cells, bs), bs, 0, s>>>(m, a); break;
        }
    }
    static bool diff_pair(const DevMesh &m, const void *inA, void *outA, const void *inB, void *outB, cudaStream_t s,
                          bool dry)
    {
        constexpr unsigned ra = out_rec_bytes<2>(), rb = out_rec_bytes<1>();
        if constexpr (ra % 16 != 0 || rb % 16 != 0) {
            return false;
        } else {
            if (dry) return true;
            constexpr int CB = 64;
            // bulk precisions fit 8 blocks per SM (64 registers, no spills); FP64 does not
            constexpr int MINB = PREC == PREC_F64 ? 1 : 8;
            k_diff_dual<DIM, NV, 2, PREC, CB, MINB><<<nblk(m.n_cells, CB), 2 * CB, (size_t)CB * (ra + rb), s>>>(
                m, inA, outA, inB, outB);
            return true;
        }
    }
    static void faces(const DevMesh &m, const StageArgs &a, double *fL, double *fR, cudaStream_t s)
    {
        k_faces<DIM, NV, NS, PREC><<<nblk(m.n_faces, 128), 128, 0, s>>>(m, a, fL, fR);
    }
    static void bnd_grad(const DevMesh &m, const void *o0, void *o1, cudaStream_t s)
    {
        if (m.n_bcell > 0) k_bnd_grad<DIM, NV, PREC><<<nblk(m.n_bcell, 128), 128, 0, s>>>(m, o0, o1);
    }
    static PathFns fns() { return PathFns{&pack, &diff, &diff_pair, &stage, &faces, &bnd_grad}; }
};

// Persistent batched stage (k_batch_stage), launched cooperatively.
struct BatchFns {
    cudaError_t (*launch)(const DevMesh &, const StageArgs &, const BatchArgs &, int grid, int block, cudaStream_t);
    int (*blocks_per_sm)(int block);
};

template <int DIM, int NV, int NS, int PREC> struct BatchPath {
    static cudaError_t launch(const DevMesh &m, const StageArgs &a, const BatchArgs &b, int grid, int block,
                              cudaStream_t s)
    {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(block);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, k_batch_stage<DIM, NV, NS, PREC>, m, a, b);
    }
    static int blocks_per_sm(int block)
    {
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_stage<DIM, NV, NS, PREC>, block, 0);
        return n;
    }
    static BatchFns fns() { return BatchFns{&launch, &blocks_per_sm}; }
};

// batch table index: dim (2,3) x nv-class x NS (1, 2) x precision
inline int batch_index(int dim, int nv, int ns, int prec) { return (((dim - 2) * 2 + (nv == 1 ? 0 : 1)) * 2 + (ns - 1)) * 3 + prec; }
constexpr int N_BATCH = 2 * 2 * 2 * 3;
void register_batch(BatchFns *t);

// table index: dim (2,3) x nv-class (scalar, Euler) x NS (1..4) x precision (3)
inline int path_index(int dim, int nv, int ns, int prec)
{
    return (((dim - 2) * 2 + (nv == 1 ? 0 : 1)) * 4 + (ns - 1)) * 3 + prec;
}
constexpr int N_PATHS = 2 * 2 * 4 * 3;

void register_paths_d2s(PathFns *t);
void register_paths_d2e(PathFns *t);
void register_paths_d3s(PathFns *t);
void register_paths_d3e(PathFns *t);

}  // namespace dol
