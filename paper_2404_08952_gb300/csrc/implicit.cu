// Semi-implicit DOLINC step for linear advection (Sec 2.4): matrix rows from the
// DOLINC weights, and one persistent cooperative launch per linear solve.
//
// k_imp_assemble  one thread per cell: for each face slot the flux speed a.S and the
//                 weights of the upwind and downwind averages in the face value
//                 (W0[0], W1[0] of the DOLINC representation, the same routine the
//                 stage kernels use), summed into the diagonal or stored against the
//                 neighbour; then every row is scaled by its diagonal.
// k_imp_solve     BiCGSTAB on the scaled rows, all iterations in one launch.  Each
//                 iteration is three grid-stride phases, each ended by a grid barrier
//                 that also reduces the phase's dot products:
//                   A  v = A p (the neighbours' p gathered);           sum rh.v
//                   B  s = r - alpha v, t = A s (the neighbours' s formed from their
//                      r and v);                      sums t.s, t.t, rh.s, rh.t
//                   C  x += alpha p + omega s; r = s - omega t;
//                      p = r + beta (p - omega v), own values only;   sum r.r
//                 omega = t.s / t.t, the next rh.r = rh.s - omega rh.t and beta come
//                 from B's sums, so C can update p without another barrier, and a
//                 neighbour is gathered three times per iteration (p; r, v).
//                 The block that arrives last at a barrier sums the per-block partials
//                 in block order (the result does not depend on arrival order),
//                 computes the next scalars and releases the grid.  A wait polls at
//                 most spin_limit times; one that gives up sets status bit 1 and an
//                 abort word that ends the solve in every block.  The launch is
//                 cooperative, so all blocks are resident and the waits end.
//                 Warm start: x starts from the previous step's solution, or from the
//                 linear extrapolation of the last two (r = b - A x0, one extra
//                 product in the set-up phase); else from 0.
//                 Vectors written inside the launch are read with ld.global.cg (L2),
//                 never through the incoherent L1.  Rows per face slot (the default:
//                 a thread's consecutive slot entries share L1 sectors) or in ELL form
//                 (width 4, 6 or 8, padded with zero weights: coalesced row loads, no
//                 reuse; measured no faster on the hex/prism mesh).
#include "common.cuh"
#include "implicit.cuh"

namespace dol {

// ----------------------------------------------------------------------------- assembly
template <int NS>
__global__ void __launch_bounds__(256) k_imp_assemble(DevMesh m, int k, int r, double ax, double ay, double az,
                                                      double inv_dt, double theta, int ell, int32_t *nbr, double *off,
                                                      double *diag, double *bscale)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m.n_cells) return;
    const long long n = m.n_cells;
    const double V = 1.0 / m.cellk64[4ll * c + 3];
    double dsum = 0.0;
    const int s0 = m.off[c], s1 = m.off[c + 1];
    // entry of slot s: ELL position (s - s0) n + c, or the slot itself (CSR)
    auto at = [&](int s) { return ell ? (long long)(s - s0) * n + c : (long long)s; };
    for (int s = s0; s < s1; ++s) {
        const int2 sw = m.slot2[s];
        const unsigned word = (unsigned)sw.y;
        const int f = (int)(word >> 2);
        const bool bnd = (word & 2u) != 0;
        const int side = (int)(word & 1u);
        const double *fr = m.face64 + 8ll * f;
        // a.S of the face in its internal owner -> neighbour orientation
        const double an = ax * fr[4] + ay * fr[5] + (m.dim == 3 ? az * fr[6] : 0.0);
        nbr[at(s)] = sw.x;
        if (bnd) {            // zero-gradient face: the flux of the cell's own value
            dsum += theta * an;
            off[at(s)] = 0.0;
            continue;
        }
        // weights of the owner's (cP) and the neighbour's (cN) averages in the upwind value
        double W0[NS + 1], W1[NS + 1], cP, cN;
        if (an >= 0.0) {
            dolinc_weights<NS, double>(k, r, fr[3], W0, W1);
            cP = W0[0];
            cN = W1[0];
        } else {
            dolinc_weights<NS, double>(k, r, rcp_bulk(fr[3]), W0, W1);
            cP = W1[0];
            cN = W0[0];
        }
        // the flux an (cP u_P + cN u_N) leaves the owner and enters the neighbour
        if (side == 0) {
            dsum += theta * an * cP;
            off[at(s)] = theta * an * cN;
        } else {
            dsum -= theta * an * cN;
            off[at(s)] = -theta * an * cP;
        }
    }
    const double D = V * inv_dt + dsum;
    const double iD = 1.0 / D;
    for (int s = s0; s < s1; ++s) off[at(s)] *= iD;
    for (int q = s1 - s0; q < ell; ++q) {      // ELL padding: the cell itself, weight 0
        nbr[(long long)q * n + c] = c;
        off[(long long)q * n + c] = 0.0;
    }
    diag[c] = D;
    bscale[c] = V * iD;
}

void launch_imp_assemble(const DevMesh &m, int ns, int k, int r, double ax, double ay, double az, double dt,
                         double theta, int ell, int32_t *nbr, double *off, double *diag, double *bscale,
                         cudaStream_t s)
{
    const int grid = (m.n_cells + 255) / 256;
    if (grid == 0) return;
    const double idt = 1.0 / dt;
    switch (ns) {
    case 1: k_imp_assemble<1><<<grid, 256, 0, s>>>(m, k, r, ax, ay, az, idt, theta, ell, nbr, off, diag, bscale); break;
    case 2: k_imp_assemble<2><<<grid, 256, 0, s>>>(m, k, r, ax, ay, az, idt, theta, ell, nbr, off, diag, bscale); break;
    case 3: k_imp_assemble<3><<<grid, 256, 0, s>>>(m, k, r, ax, ay, az, idt, theta, ell, nbr, off, diag, bscale); break;
    default: k_imp_assemble<4><<<grid, 256, 0, s>>>(m, k, r, ax, ay, az, idt, theta, ell, nbr, off, diag, bscale); break;
    }
}

// -------------------------------------------------------------------------------- solve
// Sum over the block of N values, in a fixed order; the results are in thread 0.
template <int N>
__device__ __forceinline__ void block_sum(double (&v)[N], double (*sh)[IMP_BLOCK / 32])
{
#pragma unroll
    for (int k = 0; k < N; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0)
#pragma unroll
        for (int k = 0; k < N; ++k) sh[k][w] = v[k];
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            v[k] = l < IMP_BLOCK / 32 ? sh[k][l] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
        }
    }
    __syncthreads();
}

__device__ __forceinline__ double ldcg(const double *p) { return __ldcg(p); }
__device__ __forceinline__ void stcg(double *p, double v) { __stcg(p, v); }

// Grid barrier that reduces v[0..N) over all threads of the grid.  The last block to
// arrive sums the per-block partials in block order and calls fin(sums) in its thread
// 0 (fin writes the next scalars) before the others are released.  Returns false when
// the solve was aborted (a wait gave up here or in an earlier barrier).
template <int N> struct Red {
    double v[N];
};

template <int N, class Fin>
__device__ __forceinline__ bool reduce_barrier(const ImpSolve &a, Red<N> r, Fin fin)
{
    static_assert(N <= IMP_NRED, "partials hold IMP_NRED values per block");
    double (&v)[N] = r.v;
    __shared__ double sh[N][IMP_BLOCK / 32];
    __shared__ int last, ok;
    block_sum<N>(v, sh);
    volatile unsigned *gen = a.bar + 32, *abort = a.bar + 64;
    unsigned g = 0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) a.part[IMP_NRED * blockIdx.x + k] = v[k];
        g = *gen;
        __threadfence();
        last = atomicAdd(a.bar, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
        __threadfence();
        double t[N];
#pragma unroll
        for (int k = 0; k < N; ++k) t[k] = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += IMP_BLOCK)
#pragma unroll
            for (int k = 0; k < N; ++k) t[k] += ldcg(a.part + IMP_NRED * b + k);
        block_sum<N>(t, sh);
        if (threadIdx.x == 0) {
            fin(t);
            atomicExch(a.bar, 0u);
            __threadfence();
            atomicAdd(const_cast<unsigned *>(gen), 1u);
        }
    } else if (threadIdx.x == 0) {
        unsigned it = 0;
        while (*gen == g && !*abort) {
            if (++it > a.spin_limit) {
                atomicOr(a.status, 2u);
                atomicExch(const_cast<unsigned *>(abort), 1u);
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
    }
    if (threadIdx.x == 0) ok = !*abort;
    __syncthreads();
    return ok;
}

// a.off . f(neighbour) over the row of cell c, added to acc: ELL rows of W entries
// (entry q of cell c at q n + c: a warp's loads are contiguous and independent), or the
// cell's slot range (W = 0).
template <int W, class F>
__device__ __forceinline__ double row_sum(const ImpSolve &a, int c, double acc, F f)
{
    if constexpr (W > 0) {
        int j[W];
        double o[W];
#pragma unroll
        for (int q = 0; q < W; ++q) {
            j[q] = __ldg(a.nbr + (long long)q * a.n + c);
            o[q] = __ldg(a.off + (long long)q * a.n + c);
        }
#pragma unroll
        for (int q = 0; q < W; ++q) acc = fma(o[q], f(j[q]), acc);
    } else {
        const int s0 = __ldg(a.row + c), s1 = __ldg(a.row + c + 1);
#pragma unroll 2
        for (int s = s0; s < s1; ++s) acc = fma(__ldg(a.off + s), f(__ldg(a.nbr + s)), acc);
    }
    return acc;
}

template <int W>
__global__ void __launch_bounds__(IMP_BLOCK) k_imp_solve(ImpSolve a)
{
    const int n = a.n;
    const int nth = gridDim.x * IMP_BLOCK;
    const int t0 = blockIdx.x * IMP_BLOCK + threadIdx.x;
    double *sc = a.scal;
    double *p = a.p, *v = a.v;
    bool ok;

    // Set-up: b = bscale * rhs; the initial guess x0 = 0, the previous step's solution
    // x1 (warm 1), or 2 x1 - x2 (warm 2: linear extrapolation from the last two steps),
    // formed for the neighbours on the fly and written to x; r = rh = p = b - A x0.
    {
        Red<2> red{{0.0, 0.0}};
        for (int c = t0; c < n; c += nth) {
            double rhs = a.R[c];
            if (a.Rn) rhs = (a.un[c] - a.u[c]) * a.inv_dt + a.theta * rhs + (1.0 - a.theta) * a.Rn[c];
            const double b = a.bscale[c] * rhs;
            double r0 = b, x0 = 0.0;
            if (a.warm) {
                auto guess = [&](int j) { return a.warm == 2 ? fma(2.0, a.x1[j], -a.x2[j]) : a.x1[j]; };
                x0 = guess(c);
                r0 = b - row_sum<W>(a, c, x0, guess);
            }
            a.x[c] = x0;
            a.r[c] = r0;
            a.rh[c] = r0;
            p[c] = r0;
            red.v[0] = fma(b, b, red.v[0]);
            red.v[1] = fma(r0, r0, red.v[1]);
        }
        ok = reduce_barrier(a, red, [&](const double *t) {
            stcg(sc + SC_RHO, t[1]);
            stcg(sc + SC_BB, t[0]);
            stcg(sc + SC_RR, t[1]);
            stcg(sc + SC_BRK, 0.0);
            stcg(sc + SC_SOLVES, ldcg(sc + SC_SOLVES) + 1.0);
            stcg(a.life + 1, ldcg(a.life + 1) + 1.0);
            stcg(sc + SC_DONE, (t[1] <= a.tol2 * t[0]) ? 1.0 : 0.0);
        });
    }

    for (int it = 0; ok && ldcg(sc + SC_DONE) == 0.0; ++it) {
        // A: v = A p (the neighbours' p gathered);  sum rh.v
        {
            Red<1> red{{0.0}};
            for (int c = t0; c < n; c += nth) {
                const double acc = row_sum<W>(a, c, ldcg(p + c), [&](int j) { return ldcg(p + j); });
                v[c] = acc;
                red.v[0] = fma(ldcg(a.rh + c), acc, red.v[0]);
            }
            ok = reduce_barrier(a, red, [&](const double *t) {
                if (t[0] == 0.0 || !isfinite(t[0])) {
                    atomicOr(a.status, 4u);
                    stcg(sc + SC_DONE, 1.0);
                } else {
                    stcg(sc + SC_ALPHA, ldcg(sc + SC_RHO) / t[0]);
                }
            });
            if (!ok || ldcg(sc + SC_DONE) != 0.0) break;
        }
        // B: s = r - alpha v; t = A s, the neighbours' s formed from their r and v;
        //    sums t.s, t.t, rh.s, rh.t: omega = t.s / t.t, the next rh.r = rh.s - omega
        //    rh.t, and beta, all known before the updates of phase C
        {
            const double al = ldcg(sc + SC_ALPHA);
            Red<4> red{{0.0, 0.0, 0.0, 0.0}};
            for (int c = t0; c < n; c += nth) {
                const double scv = fma(-al, ldcg(v + c), ldcg(a.r + c));
                const double acc = row_sum<W>(a, c, scv, [&](int j) { return fma(-al, ldcg(v + j), ldcg(a.r + j)); });
                a.s[c] = scv;
                a.t[c] = acc;
                const double rh = ldcg(a.rh + c);
                red.v[0] = fma(acc, scv, red.v[0]);
                red.v[1] = fma(acc, acc, red.v[1]);
                red.v[2] = fma(rh, scv, red.v[2]);
                red.v[3] = fma(rh, acc, red.v[3]);
            }
            ok = reduce_barrier(a, red, [&](const double *t) {
                stcg(sc + SC_ITERS, ldcg(sc + SC_ITERS) + 1.0);
                stcg(a.life, ldcg(a.life) + 1.0);
                const double om = t[1] > 0.0 ? t[0] / t[1] : 0.0;     // t = 0: s = 0, the next r is 0
                const double rho1 = t[2] - om * t[3];
                stcg(sc + SC_OMEGA, om);
                if (t[1] > 0.0 && (om == 0.0 || rho1 == 0.0 || !isfinite(rho1))) {
                    stcg(sc + SC_BRK, 1.0);      // breakdown: stop after phase C's updates
                    stcg(sc + SC_BETA, 0.0);
                } else {
                    stcg(sc + SC_BETA, om != 0.0 ? (rho1 / ldcg(sc + SC_RHO)) * (ldcg(sc + SC_ALPHA) / om) : 0.0);
                }
                stcg(sc + SC_RHO, rho1);
            });
            if (!ok) break;
        }
        // C: x += alpha p + omega s; r = s - omega t; p = r + beta (p - omega v), all
        //    of the cell's own values;  sum r.r (the true recursive residual)
        {
            const double al = ldcg(sc + SC_ALPHA), om = ldcg(sc + SC_OMEGA), beta = ldcg(sc + SC_BETA);
            Red<1> red{{0.0}};
            for (int c = t0; c < n; c += nth) {
                const double sv = ldcg(a.s + c), pc = ldcg(p + c);
                a.x[c] = fma(om, sv, fma(al, pc, ldcg(a.x + c)));
                const double rv = fma(-om, ldcg(a.t + c), sv);
                a.r[c] = rv;
                p[c] = fma(beta, pc - om * ldcg(v + c), rv);
                red.v[0] = fma(rv, rv, red.v[0]);
            }
            ok = reduce_barrier(a, red, [&](const double *t) {
                stcg(sc + SC_RR, t[0]);
                if (t[0] <= a.tol2 * ldcg(sc + SC_BB)) {
                    stcg(sc + SC_DONE, 1.0);
                } else if (ldcg(sc + SC_BRK) != 0.0 || !isfinite(t[0])) {
                    atomicOr(a.status, 4u);
                    stcg(sc + SC_DONE, 1.0);
                } else if (it + 1 >= a.max_iter) {
                    atomicOr(a.status, 8u);
                    stcg(sc + SC_DONE, 1.0);
                }
            });
        }
    }
    if (!ok) return;
    // u += delta
    for (int c = t0; c < n; c += nth) a.u[c] += ldcg(a.x + c);
}

template <int W> cudaError_t launch_w(const ImpSolve &a, int grid, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(IMP_BLOCK);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_imp_solve<W>, a);
}

template <int W> int blocks_w()
{
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_imp_solve<W>, IMP_BLOCK, 0);
    return n;
}

int imp_ell_width(int max_slots) { return max_slots <= 4 ? 4 : max_slots <= 6 ? 6 : max_slots <= 8 ? 8 : 0; }

cudaError_t launch_imp_solve(const ImpSolve &a, int ell, int grid, cudaStream_t s)
{
    switch (ell) {
    case 4: return launch_w<4>(a, grid, s);
    case 6: return launch_w<6>(a, grid, s);
    case 8: return launch_w<8>(a, grid, s);
    default: return launch_w<0>(a, grid, s);
    }
}

int imp_solve_blocks_per_sm(int ell)
{
    switch (ell) {
    case 4: return blocks_w<4>();
    case 6: return blocks_w<6>();
    case 8: return blocks_w<8>();
    default: return blocks_w<0>();
    }
}

}  // namespace dol
