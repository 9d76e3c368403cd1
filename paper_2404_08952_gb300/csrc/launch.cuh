// Host launchers of the templated stage kernels and the table the C ABI dispatches on.
#pragma once
#include "kernels.cuh"

namespace dol {

// Launch shape of the gather kernels: lanes per cell (1, 4 or 8) and block size.
struct Tune {
    int diff_lpc = 4, diff_block = 256, stage_lpc = 4, stage_block = 128;
};

struct PathFns {
    void (*pack)(const DevMesh &, const double *, void *, cudaStream_t);
    void (*diff)(const DevMesh &, int M, const void *, void *, const Tune &, cudaStream_t);
    void (*stage)(const DevMesh &, const StageArgs &, const Tune &, cudaStream_t);
    void (*faces)(const DevMesh &, const StageArgs &, double *, double *, cudaStream_t);
};

inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

template <int DIM, int NV, int NS, int PREC> struct Path {
    static void pack(const DevMesh &m, const double *u, void *o0, cudaStream_t s)
    {
        k_pack<NV, PREC><<<nblk(m.n_cells, 256), 256, 0, s>>>(m.n_cells, u,
                                                              static_cast<typename PrecT<PREC>::T0 *>(o0));
    }
    template <int LPC> static void diff_l(const DevMesh &m, int M, const void *in, void *out, int bs, cudaStream_t s)
    {
        const int b = nblk((long long)m.n_cells * LPC, bs);
        switch (M) {
        case 1: k_diff<DIM, NV, 1, PREC, LPC><<<b, bs, 0, s>>>(m, in, out); break;
        case 2: k_diff<DIM, NV, 2, PREC, LPC><<<b, bs, 0, s>>>(m, in, out); break;
        case 3: k_diff<DIM, NV, 3, PREC, LPC><<<b, bs, 0, s>>>(m, in, out); break;
        case 4: k_diff<DIM, NV, 4, PREC, LPC><<<b, bs, 0, s>>>(m, in, out); break;
        default: break;
        }
    }
    static void diff(const DevMesh &m, int M, const void *in, void *out, const Tune &t, cudaStream_t s)
    {
        switch (t.diff_lpc) {
        case 4: diff_l<4>(m, M, in, out, t.diff_block, s); break;
        case 8: diff_l<8>(m, M, in, out, t.diff_block, s); break;
        default: diff_l<1>(m, M, in, out, t.diff_block, s); break;
        }
    }
    static void stage(const DevMesh &m, const StageArgs &a, const Tune &t, cudaStream_t s)
    {
        const int bs = t.stage_block;
        switch (t.stage_lpc) {
        case 4: k_stage<DIM, NV, NS, PREC, 4><<<nblk((long long)m.n_cells * 4, bs), bs, 0, s>>>(m, a); break;
        case 8: k_stage<DIM, NV, NS, PREC, 8><<<nblk((long long)m.n_cells * 8, bs), bs, 0, s>>>(m, a); break;
        default: k_stage<DIM, NV, NS, PREC, 1><<<nblk(m.n_cells, bs), bs, 0, s>>>(m, a); break;
        }
    }
    static void faces(const DevMesh &m, const StageArgs &a, double *fL, double *fR, cudaStream_t s)
    {
        k_faces<DIM, NV, NS, PREC><<<nblk(m.n_faces, 128), 128, 0, s>>>(m, a, fL, fR);
    }
    static PathFns fns() { return PathFns{&pack, &diff, &stage, &faces}; }
};

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
