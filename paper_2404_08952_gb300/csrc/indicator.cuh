// Troubled-cell indicator: the criterion, the network inputs, and the network itself.
//
// The paper has no troubled-cell criterion or network; both are built from the
// paper's own quantities (the ENO3-DOLINC indicators of Sec 2.4 and the DOLINC
// differentials of Sec 2.3) and decide where ENO3-DOLINC replaces the fixed stencil.
#pragma once
#include "launch.cuh"

namespace dol {

constexpr int MLP_IN = 24, MLP_H = 64;
constexpr int MLP_PARAMS = MLP_H * MLP_IN + MLP_H + 2 * (MLP_H * MLP_H + MLP_H) + MLP_H + 1;   // 9985
// offsets of the parameter blocks in the flat vector W1 b1 W2 b2 W3 b3 W4 b4
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + MLP_H * MLP_IN, OFF_W2 = OFF_B1 + MLP_H, OFF_B2 = OFF_W2 + MLP_H * MLP_H,
              OFF_W3 = OFF_B2 + MLP_H, OFF_B3 = OFF_W3 + MLP_H * MLP_H, OFF_W4 = OFF_B3 + MLP_H,
              OFF_B4 = OFF_W4 + MLP_H;
// tensor-core B fragments (mma m16n8k16): layer 1 2x8 tiles, layers 2-3 4x8, layer 4 4x1
constexpr int FRAG_L1 = 0, FRAG_L2 = 16, FRAG_L3 = 48, FRAG_L4 = 80, N_FRAGS = 84;

struct IndicatorFns {
    void (*criterion)(const DevMesh &, const StageArgs &, double kappa, double eps, uint8_t *flags, cudaStream_t);
    void (*own_features)(const DevMesh &, const StageArgs &, float *own, cudaStream_t);
};

// table index: dim (2,3) x NSR (2..4) x precision (3)
inline int indicator_index(int dim, int nsr, int prec) { return ((dim - 2) * 3 + (nsr - 2)) * 3 + prec; }
constexpr int N_INDICATOR = 2 * 3 * 3;
void register_indicator(IndicatorFns *t);

// launchers of the precision-independent kernels (indicator.cu)
void launch_gather24(const DevMesh &m, const float *own, float *x, cudaStream_t s);
void launch_mlp_frags(const float *theta, uint2 *frag, cudaStream_t s);
void launch_mlp_infer(const uint2 *frag, const float *theta, const float *x, long long n, float *logits,
                      uint8_t *flags, cudaStream_t s);
// the network on every cell of m, its inputs gathered from the own features inside the kernel
void launch_mlp_infer_fused(const uint2 *frag, const float *theta, const DevMesh &m, const float *own, float *logits,
                            uint8_t *flags, cudaStream_t s);
void launch_quantize(const float *theta, float *theta_q, cudaStream_t s);
void launch_dense_fwd(const float *A, int in_dim, const float *W, const float *b, int out_dim, long long n, float *Z,
                      bool relu, cudaStream_t s);
void launch_dense_bwd_w(const float *dZ, const float *A, int in_dim, int out_dim, long long n, float *dW, float *db,
                        cudaStream_t s);
void launch_dense_bwd_x(const float *dZ, const float *W, int in_dim, int out_dim, long long n, const float *Amask,
                        float *dA, cudaStream_t s);
void launch_bce(const float *z, const uint8_t *y, long long n, float pos_weight, float *dz, float *loss,
                cudaStream_t s);
void launch_adam(float *theta, float *m, float *v, const float *g, int n, float lr, int step, cudaStream_t s);

}  // namespace dol
