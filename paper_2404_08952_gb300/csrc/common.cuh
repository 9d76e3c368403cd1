// Device building blocks of the DOLINC stage kernels (arXiv 2404.08952).
//
// Differentials are stored per cell as the coefficients of the homogeneous
// polynomial  p_m(d) = T^(m) : d^m  (one coefficient per monomial of degree m), so a
// 3D order-m tensor costs (m+1)(m+2)/2 numbers instead of 3^m.  Only the symmetric
// part of T^(m) reaches a face (the face contracts it with d^m), and the Gauss step
// of Sec 2.3 acts on the polynomial as a product with the linear form (S.d):
//   p_m(d) = (1/V) sum_f (S_f . d) [w p_{m-1,c}(d) + (1-w) p_{m-1,nb}(d)].
// Monomial q of degree m is d_x^a d_y^b d_z^c with t = b+c, q = t(t+1)/2 + c (3D), or
// d_x^a d_y^b with q = b (2D); this index does not depend on m.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#define DOL_HD __host__ __device__ __forceinline__

namespace dol {

constexpr int MAXN = 4;                  // highest differential order
constexpr int MAXK = 2 * MAXN + 2;       // widest stencil

DOL_HD constexpr int ncoef(int dim, int m) { return dim == 2 ? m + 1 : (m + 1) * (m + 2) / 2; }

// storage stride (elements) of a per-cell record of n elements of `bytes` each:
// padded to 16 bytes for vector loads, except tiny records.
DOL_HD constexpr int rec_stride(int n, int bytes)
{
    return (n * bytes <= 8) ? n : ((n * bytes + 15) / 16) * 16 / bytes;
}

template <class T> struct ElemBytes { static constexpr int v = sizeof(T); };

// ------------------------------------------------------------------ scalar conversion
template <class R> DOL_HD R cvt(double x) { return (R)x; }
template <class R> DOL_HD R cvt(float x) { return (R)x; }
template <class R> __device__ __forceinline__ R cvt(__nv_bfloat16 x) { return (R)__bfloat162float(x); }
template <class T, class R> __device__ __forceinline__ T to_store(R x) { return (T)x; }

// Reciprocal and square root of the bulk arithmetic.  FP64 keeps the correctly rounded
// operations; FP32 uses the PTX approximate forms (rcp.approx: <= 1 ulp, sqrt.approx:
// relative error ~2^-23), below the FP32 path's own rounding of the face values.
template <class R> __device__ __forceinline__ R rcp_bulk(R x) { return (R)1 / x; }
template <> __device__ __forceinline__ float rcp_bulk<float>(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
template <class R> __device__ __forceinline__ R sqrt_bulk(R x) { return sqrt(x); }
template <> __device__ __forceinline__ float sqrt_bulk<float>(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
template <> __device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16, float>(float x) { return __float2bfloat16_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16, double>(double x) { return __float2bfloat16_rn((float)x); }

// ------------------------------------------------------------------ record load/store
// Loads the first N elements of a record of stride S (elements of T) into registers.
// LDG: read through the read-only data path (global memory only); otherwise a generic
// load that also serves shared memory.
template <bool LDG, class V> __device__ __forceinline__ V ldv(const V *p)
{
    if constexpr (LDG) return __ldg(p);
    else return *p;
}

// 32 bytes at a 32-byte aligned global address through the read-only path (one
// 256-bit load)
__device__ __forceinline__ void ldg32(const void *p, unsigned *w)
{
    asm("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
        : "l"(p));
}

template <class T, int N, int S, class R, bool LDG = true>
__device__ __forceinline__ void load_rec(const T *__restrict__ base, long long cell, R *out)
{
    const T *p = base + cell * (long long)S;
    constexpr int B = S * (int)sizeof(T);
    if constexpr (LDG && B % 32 == 0) {
        // records of whole 32-byte chunks (record arrays start 256-byte aligned)
        constexpr int V = 32 / (int)sizeof(T);
        constexpr int NV = (N + V - 1) / V;
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            unsigned w[8];
            ldg32(p + i * V, w);
            const T *e = reinterpret_cast<const T *>(w);
#pragma unroll
            for (int j = 0; j < V; ++j)
                if (i * V + j < N) out[i * V + j] = cvt<R>(e[j]);
        }
    } else if constexpr (B % 16 == 0) {
        constexpr int V = 16 / (int)sizeof(T);
        constexpr int NV = (N + V - 1) / V;
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            uint4 q = ldv<LDG>(reinterpret_cast<const uint4 *>(p) + i);
            const T *e = reinterpret_cast<const T *>(&q);
#pragma unroll
            for (int j = 0; j < V; ++j)
                if (i * V + j < N) out[i * V + j] = cvt<R>(e[j]);
        }
    } else if constexpr (B % 8 == 0 && sizeof(T) <= 8) {
        constexpr int V = 8 / (int)sizeof(T);
        constexpr int NV = (N + V - 1) / V;
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            uint2 q = ldv<LDG>(reinterpret_cast<const uint2 *>(p) + i);
            const T *e = reinterpret_cast<const T *>(&q);
#pragma unroll
            for (int j = 0; j < V; ++j)
                if (i * V + j < N) out[i * V + j] = cvt<R>(e[j]);
        }
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) out[i] = cvt<R>(ldv<LDG>(p + i));
    }
}

// 32 bytes to a 32-byte aligned global address (one 256-bit store)
__device__ __forceinline__ void stg32(void *p, const unsigned *w)
{
    asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(w[0]), "r"(w[1]),
                 "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
                 : "memory");
}

// Stores N elements (padding lanes written as zero) of a record of stride S to global
// memory (record arrays start 256-byte aligned).
template <class T, int N, int S, class R>
__device__ __forceinline__ void store_rec(T *__restrict__ base, long long cell, const R *in)
{
    T *p = base + cell * (long long)S;
    constexpr int B = S * (int)sizeof(T);
    if constexpr (B % 32 == 0) {
        constexpr int V = 32 / (int)sizeof(T);
#pragma unroll
        for (int i = 0; i < S / V; ++i) {
            unsigned w[8];
            T *e = reinterpret_cast<T *>(w);
#pragma unroll
            for (int j = 0; j < V; ++j) e[j] = (i * V + j < N) ? to_store<T, R>(in[i * V + j]) : to_store<T, R>((R)0);
            stg32(p + i * V, w);
        }
    } else if constexpr (B % 16 == 0) {
        constexpr int V = 16 / (int)sizeof(T);
#pragma unroll
        for (int i = 0; i < S / V; ++i) {
            uint4 q;
            T *e = reinterpret_cast<T *>(&q);
#pragma unroll
            for (int j = 0; j < V; ++j) e[j] = (i * V + j < N) ? to_store<T, R>(in[i * V + j]) : to_store<T, R>((R)0);
            reinterpret_cast<uint4 *>(p)[i] = q;
        }
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) p[i] = to_store<T, R>(in[i]);
    }
}

DOL_HD constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }

// store_rec into shared memory whose records (one per thread t, S * sizeof(T) bytes, a
// multiple of 16) are contiguous, as a bulk copy to global memory wants them.  A
// straight store would have the 8 threads of each 16-byte-per-thread store wavefront
// write records 2^k x 16 bytes apart, i.e. into the same banks; here thread t writes
// its 16-byte chunks in an order rotated by r_t, chosen so that those 8 threads always
// hit 8 distinct groups of 4 banks.  The bytes written are those of store_rec.
template <class T, int N, int S, class R>
__device__ __forceinline__ void store_rec_smem(unsigned char *base, int t, const R *in)
{
    constexpr int B = S * (int)sizeof(T);
    static_assert(B % 16 == 0, "records of whole 16-byte chunks");
    constexpr int NCH = B / 16, V = 16 / (int)sizeof(T), G = gcd_c(NCH, 8);
    uint4 q[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        T *e = reinterpret_cast<T *>(&q[c]);
#pragma unroll
        for (int j = 0; j < V; ++j) e[j] = (c * V + j < N) ? to_store<T, R>(in[c * V + j]) : to_store<T, R>((R)0);
    }
    // chunk slot (t * NCH + p) lands in bank group (t * NCH + p) mod 8: with
    // p = (j + r_t) mod NCH and r_t = (t / (8 / G)) mod NCH those are distinct over
    // any 8 consecutive t for every j
    const int r = (t / (8 / G)) % NCH;
    // rotate: q[j] <- q[(j + r) mod NCH], by the binary digits of r
#pragma unroll
    for (int b = 1; b < NCH; b <<= 1) {
        uint4 u[NCH];
#pragma unroll
        for (int j = 0; j < NCH; ++j) u[j] = q[(j + b) % NCH];
        const bool on = (r & b) != 0;
#pragma unroll
        for (int j = 0; j < NCH; ++j) q[j] = on ? u[j] : q[j];
    }
    uint4 *rec = reinterpret_cast<uint4 *>(base + (size_t)t * B);
#pragma unroll
    for (int j = 0; j < NCH; ++j) {
        int p = j + r;
        p = p >= NCH ? p - NCH : p;
        rec[p] = q[j];
    }
}

// ------------------------------------------------------------------ polynomial algebra
// acc (degree m, NVAR blocks of ncoef(DIM,m)) += (s . d) * in (degree m-1)
template <int DIM, int NVAR, int M, class R>
__device__ __forceinline__ void poly_mul_acc(R *acc, const R *in, R sx, R sy, R sz)
{
    constexpr int CI = ncoef(DIM, M - 1), CO = ncoef(DIM, M);
#pragma unroll
    for (int v = 0; v < NVAR; ++v) {
#pragma unroll
        for (int t = 0; t <= (DIM == 2 ? 0 : M - 1); ++t) {
            if constexpr (DIM == 2) {
#pragma unroll
                for (int q = 0; q < CI; ++q) {
                    R x = in[v * CI + q];
                    acc[v * CO + q] = fma(sx, x, acc[v * CO + q]);
                    acc[v * CO + q + 1] = fma(sy, x, acc[v * CO + q + 1]);
                }
            } else {
#pragma unroll
                for (int c = 0; c <= t; ++c) {
                    const int q = t * (t + 1) / 2 + c;
                    R x = in[v * CI + q];
                    acc[v * CO + q] = fma(sx, x, acc[v * CO + q]);
                    acc[v * CO + q + t + 1] = fma(sy, x, acc[v * CO + q + t + 1]);
                    acc[v * CO + q + t + 2] = fma(sz, x, acc[v * CO + q + t + 2]);
                }
            }
        }
    }
}

// monomials of degree 0..N of d, concatenated (offset of degree m = sum_{j<m} ncoef(j))
DOL_HD constexpr int ncum(int dim, int m)
{
    return m < 0 ? 0 : (dim == 2 ? (m + 1) * (m + 2) / 2 : (m + 1) * (m + 2) * (m + 3) / 6);
}

template <int DIM, int N, class R>
__device__ __forceinline__ void monomials(R dx, R dy, R dz, R *mono)
{
    mono[0] = (R)1;
#pragma unroll
    for (int m = 1; m <= N; ++m) {
        const int o = ncum(DIM, m - 1), op = ncum(DIM, m - 2);
        if constexpr (DIM == 2) {
#pragma unroll
            for (int q = 0; q < m; ++q) mono[o + q] = dx * mono[op + q];
            mono[o + m] = dy * mono[op + m - 1];
        } else {
            // t <= m-1: multiply by dx (same index); t = m: from t = m-1 by dy / dz
#pragma unroll
            for (int q = 0; q < m * (m + 1) / 2; ++q) mono[o + q] = dx * mono[op + q];
#pragma unroll
            for (int c = 0; c < m; ++c) mono[o + m * (m + 1) / 2 + c] = dy * mono[op + (m - 1) * m / 2 + c];
            mono[o + m * (m + 1) / 2 + m] = dz * mono[op + (m - 1) * m / 2 + m - 1];
        }
    }
}

// ------------------------------------------------------------------ DOLINC face weights
// For upwind cell i (n = 0) and downwind cell i+1 (n = 1) with growth rate g, returns
// W0[m], W1[m] (m = 0..NS) such that the k-th order reconstruction of Eq coeff at
// x_{i+1/2}, applied to the far-field averages inverted with Eq diffDLC, equals
//   sum_m W0[m] phi_0^(m) + W1[m] phi_1^(m)
// (the "DOLINC representation" of Sec 2.4, generalised to any stencil).
// Step 1: Eq coeff weights from the barycentric form of the Lagrange interpolant of
// the primitive at the stencil's faces (face x_{i+1/2} = 0 is node r+1).
// Step 2: the transpose of the far-field recursion moves each far cell's weight onto
// the two face cells' differentials.
template <int NS, class R>
__device__ __forceinline__ void dolinc_weights(int k, int r, R g, R *W0, R *W1)
{
    if (r == 1 && k >= 2 && k <= 4) {
        // First-order DOLINC stencils in closed form (Sec 2.4: Eq coeff on geometric
        // cells combined with Eqs lCoeffDLC1/rCoeffDLC1), G_n = 1 + g + .. + g^(n-1):
        //  (2,1):      W0 = ((2+g), 1)/G2,                       W1 = (-1, 0)/G2
        //  (3,1) USR3: W0 = (g(1+3g+g^2), g^2)/(G2 G3),          W1 = (1+g-g^2, 0)/(G2 G3)
        //  (4,1) CSR4: W0 = (-g+g^2+2g^3+3g^4+g^5, g^4)/(G3 G4), W1 = (1+3g+2g^2+g^3-g^4, -g)/(G3 G4)
        const R g2 = g * g;
#pragma unroll
        for (int m = 0; m <= NS; ++m) W0[m] = W1[m] = (R)0;
        if (k == 2) {
            const R iv = rcp_bulk((R)1 + g);
            W0[0] = ((R)2 + g) * iv;
            W0[1] = iv;
            W1[0] = -iv;
        } else if (k == 3) {
            const R iv = rcp_bulk(((R)1 + g) * ((R)1 + g + g2));
            W0[0] = g * ((R)1 + (R)3 * g + g2) * iv;
            W0[1] = g2 * iv;
            W1[0] = ((R)1 + g - g2) * iv;
        } else {
            const R g3 = g2 * g, g4 = g2 * g2;
            const R iv = rcp_bulk(((R)1 + g + g2) * ((R)1 + g + g2 + g3));
            W0[0] = (-g + g2 + (R)2 * g3 + (R)3 * g4 + g4 * g) * iv;
            W0[1] = g4 * iv;
            W1[0] = ((R)1 + (R)3 * g + (R)2 * g2 + g3 - g4) * iv;
            W1[1] = -g * iv;
        }
        return;
    }
    constexpr int KM = 2 * NS + 2;
    R gi = (R)1 / g;
    // face positions x_q = right face of cell i-r+q-1, q = 0..k
    R x[KM + 1];
    {
        // right faces of cells i+n: n >= 0 -> sum_{j=1..n} g^j ; n < 0 -> -sum_{j=n+1..0} g^j
        R pos[2 * NS + 3];  // pos[n + NS + 1], n = -(NS+1) .. NS+1
        pos[NS + 1] = (R)0;                       // n = 0
        R gp = (R)1;
#pragma unroll
        for (int n = 1; n <= NS + 1; ++n) { gp *= g; pos[NS + 1 + n] = pos[NS + n] + gp; }
        R gm = (R)1;
        pos[NS] = -(R)1;                          // n = -1
#pragma unroll
        for (int n = 2; n <= NS + 1; ++n) { gm *= gi; pos[NS + 1 - n] = pos[NS + 2 - n] - gm; }
#pragma unroll
        for (int q = 0; q <= KM; ++q) {
            int n = q - r - 1;
            int idx = n + NS + 1;
            R xv = (R)0;
#pragma unroll
            for (int a = 0; a < 2 * NS + 3; ++a)
                if (a == idx) xv = pos[a];
            x[q] = (q <= k) ? xv : (R)0;
        }
    }
    const int p = r + 1;
    // pi_q = prod_{l != q} (x_q - x_l);  L'_q(0) = -pi_p / (pi_q x_q)  (q != p)
    R pip = (R)1;
#pragma unroll
    for (int l = 0; l <= KM; ++l)
        if (l <= k && l != p) pip *= -x[l];
    R dL[KM + 1];
    R sumq = (R)0;
#pragma unroll
    for (int q = 0; q <= KM; ++q) {
        R piq = (R)1;
#pragma unroll
        for (int l = 0; l <= KM; ++l)
            if (l <= k && l != q) piq *= (x[q] - x[l]);
        R v = (q <= k && q != p) ? -pip / (piq * x[q]) : (R)0;
        dL[q] = v;
        sumq += v;
    }
#pragma unroll
    for (int q = 0; q <= KM; ++q)
        if (q == p) dL[q] = -sumq;
    // c_j = dx_j * sum_{q > j} L'_q(0); accumulate the tail sum downward
    R wt[2 * NS + 2][NS + 1];       // wt[n + NS][m], n = -NS .. NS+1
#pragma unroll
    for (int a = 0; a < 2 * NS + 2; ++a)
#pragma unroll
        for (int m = 0; m <= NS; ++m) wt[a][m] = (R)0;
    R cj[KM];
    R tail = (R)0;
#pragma unroll
    for (int j = KM - 1; j >= 0; --j) {
        tail += (j + 1 <= k) ? dL[j + 1] : (R)0;
        cj[j] = (j < k) ? tail * (x[j + 1] - x[j]) : (R)0;
    }
    // cell i-r+j sits at n = j - r, i.e. row a = j - r + NS
#pragma unroll
    for (int a = 0; a < 2 * NS + 2; ++a)
#pragma unroll
        for (int j = 0; j < KM; ++j) wt[a][0] += (j - r == a - NS) ? cj[j] : (R)0;
    // transpose of the forward recursion (n >= 2, centre n-1):
    //   phi_n^(m) = g phi_{n-2}^(m) + g^{n-1} phi_{n-1}^(m+1) + (1-g) phi_{n-1}^(m)
    R gpow[NS + 2];
    gpow[0] = (R)1;
#pragma unroll
    for (int j = 1; j <= NS + 1; ++j) gpow[j] = gpow[j - 1] * g;
#pragma unroll
    for (int n = NS + 1; n >= 2; --n) {
#pragma unroll
        for (int m = 0; m <= NS - (n - 1); ++m) {
            R w = wt[n + NS][m];
            wt[n - 2 + NS][m] = fma(g, w, wt[n - 2 + NS][m]);
            wt[n - 1 + NS][m + 1] = fma(gpow[n - 1], w, wt[n - 1 + NS][m + 1]);
            wt[n - 1 + NS][m] = fma((R)1 - g, w, wt[n - 1 + NS][m]);
        }
    }
    // transpose of the backward recursion (n <= -1, centre n+1):
    //   phi_n^(m) = [phi_{n+2}^(m) - g^{n+1} phi_{n+1}^(m+1) - (1-g) phi_{n+1}^(m)] / g
    R gneg[NS + 1];                 // gneg[j] = g^{-j}
    gneg[0] = (R)1;
#pragma unroll
    for (int j = 1; j <= NS; ++j) gneg[j] = gneg[j - 1] * gi;
#pragma unroll
    for (int n = -NS; n <= -1; ++n) {
#pragma unroll
        for (int m = 0; m <= NS + n; ++m) {
            R w = wt[n + NS][m];
            wt[n + 2 + NS][m] = fma(gi, w, wt[n + 2 + NS][m]);
            wt[n + 1 + NS][m + 1] = fma(-gneg[-n], w, wt[n + 1 + NS][m + 1]);   // g^{n+1}/g = g^n
            wt[n + 1 + NS][m] = fma(-((R)1 - g) * gi, w, wt[n + 1 + NS][m]);
        }
    }
#pragma unroll
    for (int m = 0; m <= NS; ++m) { W0[m] = wt[NS][m]; W1[m] = wt[NS + 1][m]; }
}

// Both orientations' weights: (W0f, W1f) at g and (W0r, W1r) at 1/g (the neighbour-
// upwind orientation).  For the closed-form stencils (2,1), (3,1), (4,1) the 1/g
// weights are polynomials in g over the same denominator (multiplying Eq coeff's
// closed forms through by g^(k-1) etc.), so one reciprocal serves both:
//   (2,1): W0r = ((2g+1), g) iv,  W1r = (-g, 0) iv,                 iv = 1/G2
//   (3,1): W0r = ((g^2+3g+1), g) iv,  W1r = (g(g^2+g-1), 0) iv,     iv = 1/(G2 G3)
//   (4,1): W0r = ((-g^4+g^3+2g^2+3g+1), g) iv,
//          W1r = ((g^5+3g^4+2g^3+g^2-g), -g^4) iv,                   iv = 1/(G3 G4)
template <int NS, class R>
__device__ __forceinline__ void dolinc_weights_both(int k, int r, R g, R *W0f, R *W1f, R *W0r, R *W1r)
{
    if (r == 1 && k >= 2 && k <= 4) {
#pragma unroll
        for (int m = 0; m <= NS; ++m) W0f[m] = W1f[m] = W0r[m] = W1r[m] = (R)0;
        const R g2 = g * g;
        if (k == 2) {
            const R iv = rcp_bulk((R)1 + g);
            W0f[0] = ((R)2 + g) * iv;
            W0f[1] = iv;
            W1f[0] = -iv;
            W0r[0] = ((R)2 * g + (R)1) * iv;
            W0r[1] = g * iv;
            W1r[0] = -g * iv;
        } else if (k == 3) {
            const R iv = rcp_bulk(((R)1 + g) * ((R)1 + g + g2));
            W0f[0] = g * ((R)1 + (R)3 * g + g2) * iv;
            W0f[1] = g2 * iv;
            W1f[0] = ((R)1 + g - g2) * iv;
            W0r[0] = (g2 + (R)3 * g + (R)1) * iv;
            W0r[1] = g * iv;
            W1r[0] = g * (g2 + g - (R)1) * iv;
        } else {
            const R g3 = g2 * g, g4 = g2 * g2;
            const R iv = rcp_bulk(((R)1 + g + g2) * ((R)1 + g + g2 + g3));
            W0f[0] = (-g + g2 + (R)2 * g3 + (R)3 * g4 + g4 * g) * iv;
            W0f[1] = g4 * iv;
            W1f[0] = ((R)1 + (R)3 * g + (R)2 * g2 + g3 - g4) * iv;
            W1f[1] = -g * iv;
            W0r[0] = (-g4 + g3 + (R)2 * g2 + (R)3 * g + (R)1) * iv;
            W0r[1] = g * iv;
            W1r[0] = (g4 * g + (R)3 * g4 + (R)2 * g3 + g2 - g) * iv;
            W1r[1] = -g4 * iv;
        }
        return;
    }
    dolinc_weights<NS, R>(k, r, g, W0f, W1f);
    dolinc_weights<NS, R>(k, r, rcp_bulk(g), W0r, W1r);
}

// ------------------------------------------------------------------ lane groups
// Sum of v[0..P) over the LPC lanes of an aligned group (LPC a power of two dividing
// 32), by recursive halving: on return lane j of the group holds the total of
// elements [j*P/LPC, (j+1)*P/LPC) in v[0..P/LPC).  Every lane of the warp must call it.
template <int P, int LPC, class R>
__device__ __forceinline__ void group_reduce_scatter(R *v, int lane)
{
    static_assert(P % LPC == 0, "pad the array to a multiple of the group size");
    int sz = P;
#pragma unroll
    for (int o = LPC / 2; o >= 1; o >>= 1) {
        const bool up = (lane & o) != 0;
        const int h = sz / 2;
#pragma unroll
        for (int i = 0; i < P / 2; ++i) {
            if (i < h) {
                R send = up ? v[i] : v[i + h];
                R keep = up ? v[i + h] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
        sz = h;
    }
}

// ------------------------------------------------------------------ fluxes
template <int DIM, class R>
__device__ __forceinline__ void euler_phys(R gam, const R *U, R sx, R sy, R sz, R *F, R &un, R &c2)
{
    R rho = U[0];
    R ir = rcp_bulk(rho);
    R vx = U[1] * ir, vy = U[2] * ir, vz = DIM == 3 ? U[3] * ir : (R)0;
    R ke = vx * U[1] + vy * U[2] + (DIM == 3 ? vz * U[3] : (R)0);
    R E = U[DIM + 1];
    R p = (gam - (R)1) * (E - (R)0.5 * ke);
    R vn = vx * sx + vy * sy + (DIM == 3 ? vz * sz : (R)0);
    F[0] = rho * vn;
    F[1] = U[1] * vn + p * sx;
    F[2] = U[2] * vn + p * sy;
    if constexpr (DIM == 3) F[3] = U[3] * vn + p * sz;
    F[DIM + 1] = (E + p) * vn;
    un = vn;
    c2 = gam * p * ir;
}

// Rusanov / local Lax-Friedrichs flux through S (|S| = smag)
template <int DIM, class R>
__device__ __forceinline__ void rusanov(R gam, const R *UL, const R *UR, R sx, R sy, R sz, R smag, R *F)
{
    R FL[DIM + 2], FR[DIM + 2], unL, unR, c2L, c2R;
    euler_phys<DIM, R>(gam, UL, sx, sy, sz, FL, unL, c2L);
    euler_phys<DIM, R>(gam, UR, sx, sy, sz, FR, unR, c2R);
    R a = fmax(fabs(unL) + sqrt_bulk(c2L) * smag, fabs(unR) + sqrt_bulk(c2R) * smag);
#pragma unroll
    for (int v = 0; v < DIM + 2; ++v) F[v] = (R)0.5 * (FL[v] + FR[v]) - (R)0.5 * a * (UR[v] - UL[v]);
}

}  // namespace dol
