// Semi-implicit DOLINC step for linear advection (Sec 2.4, Eq USR3 and Eq CSR4).
//
// A DOLINC face value is w_s phi_up + (1 - w_s) phi_down + c_r.  Under an implicit time
// integration the weight part is taken at the new time level and c_r (the inverted
// far-field data) stays explicit.  For a theta scheme the step in delta form is
//     (V/dt + theta K) delta = V R(u),      u' = u + delta,
// with R the explicit DOLINC residual and K the weight part of the face fluxes.  The
// rows are scaled by their diagonal, so the kernels solve
//     (I + D^-1 O) delta = D^-1 V R,    D = V/dt + theta K_cc,  O the off-diagonal part,
// stored per face slot of each cell (the slot tables of the stage kernels).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "device_mesh.hpp"

namespace dol {

// Arguments of the persistent BiCGSTAB launch.
struct ImpSolve {
    int n;                       // cells
    const int32_t *row;          // [n+1] slot ranges (the mesh's; rows without an ELL width)
    const int32_t *nbr;          // neighbour cell of each entry: ELL [W][n], else [n_slots]
    const double *off;           // its scaled off-diagonal coefficient, same layout
    const double *bscale;        // [n] V_c / D_c
    // right-hand side b_c = bscale_c * rhs_c:
    //   first solve of a step  rhs = R(u)
    //   later (outer) solves   rhs = (u_n - u)/dt + theta R(u) + (1 - theta) R(u_n)
    const double *R, *Rn, *un;   // Rn, un null on the first solve
    double inv_dt, theta;
    double *u;                   // iterate, u += delta at the end
    double *x, *r, *rh, *p, *v, *s, *t;   // [n] each
    double *part;                // [grid][IMP_NRED] per-block partial sums
    double *scal;                // solver scalars, SC_* layout
    double *life;                // [2] iterations and solves since the solver was created
    unsigned *bar;               // [0] arrivals, [32] generation, [64] abort
    unsigned *status;            // bit 1 barrier wait gave up, bit 2 breakdown, bit 3 not converged
    double tol2;                 // (relative tolerance)^2 on ||b - A x||^2 / ||b||^2
    int warm;                    // initial guess: 0 zero, 1 x1, 2 2 x1 - x2
    const double *x1, *x2;       // the previous steps' solutions (warm >= 1, warm = 2)
    int max_iter;
    unsigned spin_limit;
};

// Layout of ImpSolve::scal.  Iteration counts accumulate over the solves of a step;
// the rest describe the last solve.
enum { SC_RHO = 0, SC_ALPHA, SC_OMEGA, SC_BETA, SC_BB, SC_RR, SC_DONE, SC_ITERS, SC_SOLVES, SC_BRK, SC_COUNT };

// ELL width of the rows for cells of at most max_slots faces (4, 6, 8; 0: slot ranges)
int imp_ell_width(int max_slots);
cudaError_t launch_imp_solve(const ImpSolve &a, int ell, int grid, cudaStream_t s);
int imp_solve_blocks_per_sm(int ell);
constexpr int IMP_BLOCK = 256;
constexpr int IMP_NRED = 4;      // values a grid barrier reduces at most (partials per block)

// Rows of (V/dt + theta K): nbr, off (scaled by 1/diag), diag and bscale, in ELL form of
// width ell (padding: the cell itself with weight 0) or per slot (ell = 0).  ns: the
// scheme's needed differential order (sizes the weight arrays).
void launch_imp_assemble(const DevMesh &m, int ns, int k, int r, double ax, double ay, double az, double dt,
                         double theta, int ell, int32_t *nbr, double *off, double *diag, double *bscale,
                         cudaStream_t s);

}  // namespace dol
