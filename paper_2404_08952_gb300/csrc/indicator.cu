// Troubled-cell indicator kernels: criterion, network inputs, tensor-core inference and
// the FP32 training kernels (see indicator.cuh).
#include <cuda_bf16.h>

#include "indicator.cuh"

namespace dol {

namespace {

// ------------------------------------------------------------------ criterion
// Cell c is troubled if, at one of its interior faces, (i) a reconstructed state of
// either orientation has rho <= 0 or p <= 0, or (ii) with c upwind, the ENO3-DOLINC
// three-cell indicators of rho or rho E (Sec 2.4) satisfy
// |D_C| > kappa min(|D_L|, |D_R|) and |D_C| > eps (|phi_0| + |phi_1|).
template <int DIM, class R>
__device__ __forceinline__ R pressure_of(R gam, const R *U)
{
    R ke = U[1] * U[1] + U[2] * U[2] + (DIM == 3 ? U[3] * U[3] : (R)0);
    return (gam - (R)1) * (U[DIM + 1] - (R)0.5 * ke / U[0]);
}

template <class R>
__device__ __forceinline__ bool rough(R g, const R *p0, const R *p1, R kappa, R eps)
{
    // far values phi_{-1}, phi_{-2}, phi_2 by Eq diffDLC (c is cell i, its neighbour i+1)
    const R gi = (R)1 / g;
    const R m1_0 = gi * (p1[0] - p0[1] - ((R)1 - g) * p0[0]);
    const R m1_1 = gi * (p1[1] - p0[2] - ((R)1 - g) * p0[1]);
    const R m2 = gi * (p0[0] - gi * m1_1 - ((R)1 - g) * m1_0);
    const R p2 = g * p0[0] + g * p1[1] + ((R)1 - g) * p1[0];
    const R DL = g * g * (p0[0] - ((R)1 + g) * m1_0 + g * m2);
    const R DC = p1[0] - ((R)1 + g) * p0[0] + g * m1_0;
    const R DR = (p2 - ((R)1 + g) * p1[0] + g * p0[0]) * gi * gi;
    const R mn = fmin(fabs(DL), fabs(DR));
    return fabs(DC) > kappa * mn && fabs(DC) > eps * (fabs(p0[0]) + fabs(p1[0]));
}

template <int DIM, int NSR, int PREC>
__global__ void __launch_bounds__(128) k_criterion(DevMesh mesh, StageArgs a, float kappa, float eps, uint8_t *flags)
{
    using R = typename PrecT<PREC>::R;
    constexpr int NV = DIM + 2;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= mesh.n_cells) return;
    bool trouble = false;
    int s0, s1;
    slot_range(mesh, c, s0, s1);
    for (int s = s0; s < s1; ++s) {
        const int2 sw = __ldg(mesh.slot2 + s);
        const unsigned word = (unsigned)sw.y;
        if (word & 2) continue;                       // boundary face
        const int nb = sw.x, f = (int)(word >> 2), side = word & 1;
        R fr[8];
        {
            const R *p = Geo<R>::face(mesh) + 8ll * f;
            ld4<R>(p, fr[0], fr[1], fr[2], fr[3]);
            ld4<R>(p + 4, fr[4], fr[5], fr[6], fr[7]);
        }
        const int P = side ? nb : c, N = side ? c : nb;
        R mono[ncum(DIM, NSR)];
        monomials<DIM, NSR, R>(fr[0], fr[1], fr[2], mono);
        R phP[NV][NSR + 1], phN[NV][NSR + 1];
        contract_cell<DIM, NV, NSR, PREC>(a, P, mono, phP, mesh);
        contract_cell<DIM, NV, NSR, PREC>(a, N, mono, phN, mesh);
        const R g = fr[3];
        // (i) positivity of both reconstructed states of the face
        R W0[NSR + 1], W1[NSR + 1], UL[NV], UR[NV];
        dolinc_weights<NSR, R>(a.k, a.r, g, W0, W1);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            R t = (R)0;
#pragma unroll
            for (int m = 0; m <= NSR; ++m) t = fma(W0[m], phP[v][m], fma(W1[m], phN[v][m], t));
            UL[v] = t;
        }
        dolinc_weights<NSR, R>(a.k, a.r, (R)1 / g, W0, W1);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            R t = (R)0;
#pragma unroll
            for (int m = 0; m <= NSR; ++m) {
                R q = fma(W0[m], phN[v][m], W1[m] * phP[v][m]);
                t = (m & 1) ? t - q : t + q;
            }
            UR[v] = t;
        }
        const R gam = (R)a.gamma;
        if (!(UL[0] > (R)0) || !(pressure_of<DIM, R>(gam, UL) > (R)0) || !(UR[0] > (R)0) ||
            !(pressure_of<DIM, R>(gam, UR) > (R)0))
            trouble = true;
        // (ii) smoothness with c as the upwind cell
        const R gc = side ? (R)1 / g : g;
#pragma unroll
        for (int vi = 0; vi < 2; ++vi) {
            const int v = vi == 0 ? 0 : NV - 1;
            R q0[3], q1[3];
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const R sg = (side && (m & 1)) ? (R)-1 : (R)1;
                q0[m] = sg * (side ? phN[v][m] : phP[v][m]);
                q1[m] = sg * (side ? phP[v][m] : phN[v][m]);
            }
            if (rough<R>(gc, q0, q1, (R)kappa, (R)eps)) trouble = true;
        }
    }
    flags[c] = trouble ? 1 : 0;
}

// ------------------------------------------------------------------ network inputs
// Own features of cell c: for m = 1, 2, the largest |phi^(m)_c(d_f)| over its faces of
// rho, rho E and the momentum vector, divided by rho_c, |E_c|, sqrt(rho_c |E_c|), mapped
// by log(1 + x).
template <int DIM, int PREC>
__global__ void __launch_bounds__(128) k_own_features(DevMesh mesh, StageArgs a, float *own)
{
    using R = typename PrecT<PREC>::R;
    constexpr int NV = DIM + 2;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= mesh.n_cells) return;
    using T1 = typename OrdT<PREC, 1>::T;
    using T2 = typename OrdT<PREC, 2>::T;
    constexpr int C1 = ncoef(DIM, 1), C2 = ncoef(DIM, 2);
    R p1[NV * C1], p2[NV * C2], u0[NV];
    load_rec<typename PrecT<PREC>::T0, NV, ord_stride<DIM, NV, 0, PREC>(), R>(
        static_cast<const typename PrecT<PREC>::T0 *>(a.ord[0]), c, u0);
    load_rec<T1, NV * C1, ord_stride<DIM, NV, 1, PREC>(), R>(static_cast<const T1 *>(a.ord[1]), c, p1);
    load_rec<T2, NV * C2, ord_stride<DIM, NV, 2, PREC>(), R>(static_cast<const T2 *>(a.ord[2]), c, p2);
    R mx[6] = {0, 0, 0, 0, 0, 0};
    int s0, s1;
    slot_range(mesh, c, s0, s1);
    for (int s = s0; s < s1; ++s) {
        const int f = (int)((unsigned)__ldg(mesh.slot2 + s).y >> 2);
        R d0, d1, d2, gg;
        ld4<R>(Geo<R>::face(mesh) + 8ll * f, d0, d1, d2, gg);
        R mono[ncum(DIM, 2)];
        monomials<DIM, 2, R>(d0, d1, d2, mono);
        R ph[NV][2];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            R t1 = (R)0, t2 = (R)0;
#pragma unroll
            for (int q = 0; q < C1; ++q) t1 = fma(p1[v * C1 + q], mono[1 + q], t1);
#pragma unroll
            for (int q = 0; q < C2; ++q) t2 = fma(p2[v * C2 + q], mono[1 + C1 + q], t2);
            ph[v][0] = (R)2 * t1;
            ph[v][1] = (R)4 * t2;
        }
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            R mo = (R)0;
#pragma unroll
            for (int k = 0; k < DIM; ++k) mo += ph[1 + k][m] * ph[1 + k][m];
            mx[3 * m + 0] = fmax(mx[3 * m + 0], fabs(ph[0][m]));
            mx[3 * m + 1] = fmax(mx[3 * m + 1], fabs(ph[NV - 1][m]));
            mx[3 * m + 2] = fmax(mx[3 * m + 2], sqrt(mo));
        }
    }
    const R tiny = (R)1e-6;
    const R E = fabs(u0[NV - 1]);
    const R sc[3] = {u0[0] + tiny, E + tiny, sqrt(fabs(u0[0]) * E) + tiny};
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int q = 0; q < 3; ++q) own[6ll * c + 3 * m + q] = (float)log1p(mx[3 * m + q] / sc[q]);
}

__device__ __forceinline__ bool lex_gt(const float *a, const float *b)
{
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        if (a[q] > b[q]) return true;
        if (a[q] < b[q]) return false;
    }
    return false;
}

// Network input of cell c: its own 6 features, then the 6 of the three largest face
// neighbours in lexicographic order (itself across a boundary face).
__device__ __forceinline__ void gather24_cell(const DevMesh &mesh, const float *__restrict__ own, int c, float *o)
{
    float top[3][6];
    int have = 0;
    int s0, s1;
    slot_range(mesh, c, s0, s1);
    for (int s = s0; s < s1; ++s) {
        const int nb = __ldg(mesh.slot2 + s).x;
        float f[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) f[q] = __ldg(own + 6ll * nb + q);
        // insert into the descending top-3 list (compile-time indices only)
        bool ins0 = have < 1 || lex_gt(f, top[0]);
        bool ins1 = !ins0 && (have < 2 || lex_gt(f, top[1]));
        bool ins2 = !ins0 && !ins1 && (have < 3 || lex_gt(f, top[2]));
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            float t0 = top[0][q], t1 = top[1][q];
            if (ins0) { top[2][q] = t1; top[1][q] = t0; top[0][q] = f[q]; }
            else if (ins1) { top[2][q] = t1; top[1][q] = f[q]; }
            else if (ins2) { top[2][q] = f[q]; }
        }
        if (have < 3) ++have;
    }
    float self[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) self[q] = __ldg(own + 6ll * c + q);
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (a >= have)
#pragma unroll
            for (int q = 0; q < 6; ++q) top[a][q] = self[q];
#pragma unroll
    for (int q = 0; q < 6; ++q) o[q] = self[q];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int q = 0; q < 6; ++q) o[6 + 6 * a + q] = top[a][q];
}

__global__ void __launch_bounds__(128) k_gather24(DevMesh mesh, const float *__restrict__ own, float *__restrict__ x)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= mesh.n_cells) return;
    float o[24];
    gather24_cell(mesh, own, c, o);
#pragma unroll
    for (int q = 0; q < 24; ++q) x[24ll * c + q] = o[q];
}

// ------------------------------------------------------------------ tensor-core inference
// B fragments of mma.m16n8k16 (bf16, "col" B = W^T): lane (g = lane/4, t = lane%4) of
// tile (kt, nt) holds W[n][k], W[n][k+1] and W[n][k+8], W[n][k+9] with n = 8 nt + g,
// k = 16 kt + 2 t (zero outside the layer).
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}

__global__ void k_mlp_frags(const float *__restrict__ theta, uint2 *__restrict__ frag)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N_FRAGS * 32) return;
    const int fidx = i / 32, lane = i % 32, g = lane >> 2, t = lane & 3;
    int layer, kt, nt, in_dim, out_dim, woff;
    if (fidx < FRAG_L2) { layer = 0; kt = fidx / 8; nt = fidx % 8; in_dim = MLP_IN; out_dim = MLP_H; woff = OFF_W1; }
    else if (fidx < FRAG_L3) { layer = 1; kt = (fidx - FRAG_L2) / 8; nt = (fidx - FRAG_L2) % 8; in_dim = MLP_H; out_dim = MLP_H; woff = OFF_W2; }
    else if (fidx < FRAG_L4) { layer = 2; kt = (fidx - FRAG_L3) / 8; nt = (fidx - FRAG_L3) % 8; in_dim = MLP_H; out_dim = MLP_H; woff = OFF_W3; }
    else { layer = 3; kt = fidx - FRAG_L4; nt = 0; in_dim = MLP_H; out_dim = 1; woff = OFF_W4; }
    (void)layer;
    const int n = 8 * nt + g, k = 16 * kt + 2 * t;
    auto w = [&](int kk) { return (n < out_dim && kk < in_dim) ? theta[woff + n * in_dim + kk] : 0.0f; };
    frag[i] = make_uint2(pack_bf16(w(k), w(k + 1)), pack_bf16(w(k + 8), w(k + 9)));
}

__device__ __forceinline__ void mma_bf16(float *d, const uint32_t *a, uint2 b)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

// 16 cells per warp tile; activations stay in registers between layers (the f32
// accumulator layout of two adjacent n-tiles is the bf16 A layout of one k-tile).
// FUSED: the inputs are not read from x but gathered per tile (gather24_cell, lanes
// 0-15 one cell each) into the warp's 16 x 24 shared-memory rows.
template <bool FUSED>
__global__ void __launch_bounds__(128) k_mlp_infer(const uint2 *__restrict__ frag, const float *__restrict__ theta,
                                                   const float *__restrict__ x, long long n,
                                                   float *__restrict__ logits, uint8_t *__restrict__ flags,
                                                   DevMesh mesh, const float *__restrict__ own)
{
    __shared__ float sx[FUSED ? 4 * 16 * MLP_IN : 1];
    __shared__ uint2 sfrag[N_FRAGS * 32];
    __shared__ float sbias[3 * MLP_H + 1];
    for (int i = threadIdx.x; i < N_FRAGS * 32; i += blockDim.x) sfrag[i] = frag[i];
    for (int i = threadIdx.x; i < MLP_H; i += blockDim.x) {
        sbias[i] = __bfloat162float(__float2bfloat16_rn(theta[OFF_B1 + i]));
        sbias[MLP_H + i] = __bfloat162float(__float2bfloat16_rn(theta[OFF_B2 + i]));
        sbias[2 * MLP_H + i] = __bfloat162float(__float2bfloat16_rn(theta[OFF_B3 + i]));
    }
    if (threadIdx.x == 0) sbias[3 * MLP_H] = __bfloat162float(__float2bfloat16_rn(theta[OFF_B4]));
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const long long warps = (long long)gridDim.x * (blockDim.x / 32);
    const long long w0 = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    for (long long tile = w0; tile * 16 < n; tile += warps) {
        const long long r0 = tile * 16 + g, r1 = r0 + 8;
        float *wx = sx + (FUSED ? (threadIdx.x / 32) * 16 * MLP_IN : 0);
        if constexpr (FUSED) {
            __syncwarp();
            const long long cr = tile * 16 + lane;
            if (lane < 16 && cr < n) gather24_cell(mesh, own, (int)cr, wx + lane * MLP_IN);
            __syncwarp();
        }
        // layer 1 input: 24 features padded to 32 (two k-tiles)
        uint32_t A[4][4];
        auto xv = [&](long long r, int col) {
            if (r >= n || col >= MLP_IN) return 0.0f;
            if constexpr (FUSED) return wx[(r - tile * 16) * MLP_IN + col];
            else return __ldg(x + r * MLP_IN + col);
        };
#pragma unroll
        for (int kt = 0; kt < 2; ++kt) {
            const int c0 = 16 * kt + 2 * t;
            A[kt][0] = pack_bf16(xv(r0, c0), xv(r0, c0 + 1));
            A[kt][1] = pack_bf16(xv(r1, c0), xv(r1, c0 + 1));
            A[kt][2] = pack_bf16(xv(r0, c0 + 8), xv(r0, c0 + 9));
            A[kt][3] = pack_bf16(xv(r1, c0 + 8), xv(r1, c0 + 9));
        }
        float C[8][4];
        // three hidden layers
#pragma unroll
        for (int layer = 0; layer < 3; ++layer) {
            const int nk = layer == 0 ? 2 : 4;
            const int fbase = layer == 0 ? FRAG_L1 : (layer == 1 ? FRAG_L2 : FRAG_L3);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const float b0 = sbias[layer * MLP_H + 8 * nt + 2 * t], b1 = sbias[layer * MLP_H + 8 * nt + 2 * t + 1];
                C[nt][0] = b0; C[nt][1] = b1; C[nt][2] = b0; C[nt][3] = b1;
#pragma unroll
                for (int kt = 0; kt < 4; ++kt)
                    if (kt < nk) mma_bf16(C[nt], A[kt], sfrag[(fbase + kt * 8 + nt) * 32 + lane]);
            }
#pragma unroll
            for (int kt = 0; kt < 4; ++kt) {
                A[kt][0] = pack_bf16(fmaxf(C[2 * kt][0], 0.f), fmaxf(C[2 * kt][1], 0.f));
                A[kt][1] = pack_bf16(fmaxf(C[2 * kt][2], 0.f), fmaxf(C[2 * kt][3], 0.f));
                A[kt][2] = pack_bf16(fmaxf(C[2 * kt + 1][0], 0.f), fmaxf(C[2 * kt + 1][1], 0.f));
                A[kt][3] = pack_bf16(fmaxf(C[2 * kt + 1][2], 0.f), fmaxf(C[2 * kt + 1][3], 0.f));
            }
        }
        float O[4] = {sbias[3 * MLP_H], 0.f, sbias[3 * MLP_H], 0.f};
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) mma_bf16(O, A[kt], sfrag[(FRAG_L4 + kt) * 32 + lane]);
        if (t == 0) {
            if (r0 < n) {
                if (logits) logits[r0] = O[0];
                if (flags) flags[r0] = O[0] > 0.f;
            }
            if (r1 < n) {
                if (logits) logits[r1] = O[2];
                if (flags) flags[r1] = O[2] > 0.f;
            }
        }
    }
}

// ------------------------------------------------------------------ training (FP32)
__global__ void k_quantize(const float *__restrict__ theta, float *__restrict__ q, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) q[i] = __bfloat162float(__float2bfloat16_rn(theta[i]));
}

// Z[r][o] = b[o] + sum_i A[r][i] W[o][i]  (ReLU on request); one thread per (r, o)
__global__ void k_dense_fwd(const float *__restrict__ A, int in_dim, const float *__restrict__ W,
                            const float *__restrict__ b, int out_dim, long long n, float *__restrict__ Z, int relu)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * out_dim) return;
    const long long r = i / out_dim;
    const int o = (int)(i % out_dim);
    float s = b[o];
    for (int k = 0; k < in_dim; ++k) s = fmaf(A[r * in_dim + k], W[o * in_dim + k], s);
    Z[i] = relu ? fmaxf(s, 0.f) : s;
}

// dW[o][i] += sum_r dZ[r][o] A[r][i], db[o] += sum_r dZ[r][o]: one thread per (o, i | bias)
// and chunk of rows, atomically added (the weight gradient is a small dense array).
__global__ void k_dense_bwd_w(const float *__restrict__ dZ, const float *__restrict__ A, int in_dim, int out_dim,
                              long long n, float *__restrict__ dW, float *__restrict__ db, int chunk)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int per = in_dim + 1;
    if (j >= out_dim * per) return;
    const int o = j / per, i = j % per;
    const long long r0 = (long long)blockIdx.y * chunk;
    const long long r1 = r0 + chunk < n ? r0 + chunk : n;
    float s = 0.f;
    for (long long r = r0; r < r1; ++r) s = fmaf(dZ[r * out_dim + o], i < in_dim ? A[r * in_dim + i] : 1.f, s);
    if (i < in_dim) atomicAdd(dW + o * in_dim + i, s);
    else atomicAdd(db + o, s);
}

// dA[r][i] = (sum_o dZ[r][o] W[o][i]) * (Amask[r][i] > 0)
__global__ void k_dense_bwd_x(const float *__restrict__ dZ, const float *__restrict__ W, int in_dim, int out_dim,
                              long long n, const float *__restrict__ Amask, float *__restrict__ dA)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * in_dim) return;
    const long long r = i / in_dim;
    const int k = (int)(i % in_dim);
    float s = 0.f;
    for (int o = 0; o < out_dim; ++o) s = fmaf(dZ[r * out_dim + o], W[o * in_dim + k], s);
    dA[i] = Amask[i] > 0.f ? s : 0.f;
}

// weighted BCE with logits: dz = (s (pw y + 1 - y) - pw y) / n, loss summed into *loss
__global__ void k_bce(const float *__restrict__ z, const uint8_t *__restrict__ y, long long n, float pw,
                      float *__restrict__ dz, float *__restrict__ loss)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (i < n) {
        const float zi = z[i], yi = y[i] ? 1.f : 0.f;
        const float s = 1.f / (1.f + expf(-zi));
        dz[i] = (s * (pw * yi + 1.f - yi) - pw * yi) / (float)n;
        const float lsp = zi > 0.f ? zi + log1pf(expf(-zi)) : log1pf(expf(zi));   // log(1 + e^z)
        l = (pw * yi * (lsp - zi) + (1.f - yi) * lsp) / (float)n;
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, l);
}

__global__ void k_adam(float *theta, float *m, float *v, const float *g, int n, float lr, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi, vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

template <int DIM, int NSR, int PREC>
void crit_launch(const DevMesh &m, const StageArgs &a, double kappa, double eps, uint8_t *flags, cudaStream_t s)
{
    k_criterion<DIM, NSR, PREC><<<nblk(m.n_cells, 128), 128, 0, s>>>(m, a, (float)kappa, (float)eps, flags);
}
template <int DIM, int PREC> void own_launch(const DevMesh &m, const StageArgs &a, float *own, cudaStream_t s)
{
    k_own_features<DIM, PREC><<<nblk(m.n_cells, 128), 128, 0, s>>>(m, a, own);
}

template <int DIM, int NSR> void reg_one(IndicatorFns *t)
{
    t[indicator_index(DIM, NSR, PREC_F64)] = IndicatorFns{&crit_launch<DIM, NSR, PREC_F64>, &own_launch<DIM, PREC_F64>};
    t[indicator_index(DIM, NSR, PREC_F32)] = IndicatorFns{&crit_launch<DIM, NSR, PREC_F32>, &own_launch<DIM, PREC_F32>};
    t[indicator_index(DIM, NSR, PREC_BF16)] = IndicatorFns{&crit_launch<DIM, NSR, PREC_BF16>, &own_launch<DIM, PREC_BF16>};
}

}  // namespace

void register_indicator(IndicatorFns *t)
{
    reg_one<2, 2>(t);
    reg_one<2, 3>(t);
    reg_one<2, 4>(t);
    reg_one<3, 2>(t);
    reg_one<3, 3>(t);
    reg_one<3, 4>(t);
}

void launch_gather24(const DevMesh &m, const float *own, float *x, cudaStream_t s)
{
    k_gather24<<<nblk(m.n_cells, 128), 128, 0, s>>>(m, own, x);
}
void launch_mlp_frags(const float *theta, uint2 *frag, cudaStream_t s)
{
    k_mlp_frags<<<nblk(N_FRAGS * 32, 256), 256, 0, s>>>(theta, frag);
}
void launch_mlp_infer(const uint2 *frag, const float *theta, const float *x, long long n, float *logits,
                      uint8_t *flags, cudaStream_t s)
{
    long long tiles = (n + 15) / 16;
    int blocks = (int)((tiles + 3) / 4);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_mlp_infer<false><<<blocks, 128, 0, s>>>(frag, theta, x, n, logits, flags, DevMesh{}, nullptr);
}
void launch_mlp_infer_fused(const uint2 *frag, const float *theta, const DevMesh &m, const float *own, float *logits,
                            uint8_t *flags, cudaStream_t s)
{
    const long long n = m.n_cells;
    long long tiles = (n + 15) / 16;
    int blocks = (int)((tiles + 3) / 4);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_mlp_infer<true><<<blocks, 128, 0, s>>>(frag, theta, nullptr, n, logits, flags, m, own);
}
void launch_quantize(const float *theta, float *q, cudaStream_t s)
{
    k_quantize<<<nblk(MLP_PARAMS, 256), 256, 0, s>>>(theta, q, MLP_PARAMS);
}
void launch_dense_fwd(const float *A, int in_dim, const float *W, const float *b, int out_dim, long long n, float *Z,
                      bool relu, cudaStream_t s)
{
    k_dense_fwd<<<nblk(n * out_dim, 256), 256, 0, s>>>(A, in_dim, W, b, out_dim, n, Z, relu ? 1 : 0);
}
void launch_dense_bwd_w(const float *dZ, const float *A, int in_dim, int out_dim, long long n, float *dW, float *db,
                        cudaStream_t s)
{
    const int chunk = 2048;
    dim3 grid(nblk(out_dim * (in_dim + 1), 128), (unsigned)((n + chunk - 1) / chunk));
    k_dense_bwd_w<<<grid, 128, 0, s>>>(dZ, A, in_dim, out_dim, n, dW, db, chunk);
}
void launch_dense_bwd_x(const float *dZ, const float *W, int in_dim, int out_dim, long long n, const float *Amask,
                        float *dA, cudaStream_t s)
{
    k_dense_bwd_x<<<nblk(n * in_dim, 256), 256, 0, s>>>(dZ, W, in_dim, out_dim, n, Amask, dA);
}
void launch_bce(const float *z, const uint8_t *y, long long n, float pw, float *dz, float *loss, cudaStream_t s)
{
    k_bce<<<nblk(n, 256), 256, 0, s>>>(z, y, n, pw, dz, loss);
}
void launch_adam(float *theta, float *m, float *v, const float *g, int n, float lr, int step, cudaStream_t s)
{
    const float c1 = 1.f - powf(0.9f, (float)step), c2 = 1.f - powf(0.999f, (float)step);
    k_adam<<<nblk(n, 256), 256, 0, s>>>(theta, m, v, g, n, lr, c1, c2);
}

}  // namespace dol
