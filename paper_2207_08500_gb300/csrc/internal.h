// Internal declarations shared by the library's translation units: kernel
// parameter blocks and launcher entry points.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace neno6 {

// Classifier of Sec. 3.1: widths 6-64-32-16-8-4; parameters packed per layer
// as W[out][in] row-major followed by b[out] (the weights-file order).
constexpr int kNetWidths[6] = {6, 64, 32, 16, 8, 4};
constexpr int kNetParams = 6 * 64 + 64 + 64 * 32 + 32 + 32 * 16 + 16 + 16 * 8 + 8 + 8 * 4 + 4;
static_assert(kNetParams == 3228, "6-64-32-16-8-4 parameter count");

struct NetF64 {
  double p[kNetParams];
};

// Mask modes (public NENO6_MASK_* plus the frozen-mask mode).
enum MaskMode { kMaskMLP = 0, kMaskSmooth = 1, kMaskRough = 2, kMaskTeno = 3, kMaskGiven = 4 };

// TENO6-opt smoothness indicators (Sec. 2.1, Jiang-Shu definition): beta =
// v^T B v with v the stencil's values minus its first value; B of S0, S1, S2
// (3 x 3 each, offsets 0, 9, 18), S3 (4 x 4, offset 27) and the six-point
// stencil (6 x 6, offset 43), row-major.  Each entry is the exact rational
// value rounded once to binary64.
constexpr int kTenoTable = 79;
void teno_tables(double out[kTenoTable]);

// Arguments of one RHS / RK3-stage launch.  The tensor map (filled by
// launch_rhs_fp64) describes U as a [nv][ny][nx] float64 tensor with the box
// of one FP64 tile and its halo; use_tma = 0 when U cannot be described (odd
// nx, 1D) and every tile is loaded with plain loads.
struct RhsArgs {
  CUtensorMap tmap;
  int use_tma;
  const double* U;   // state the right-hand side is evaluated on
  const double* U0;  // state at the start of the RK3 step (stages 2, 3)
  double* out;       // dU/dt (stage 0) or the next stage state
  const uint8_t* mask_in;
  uint8_t* mask_out;
  int* status;
  const unsigned long long* smax;  // stage 1: bit patterns of max(|u|+c), max(|v|+c)
  double* dt_dev;                  // stage 1 writes, stages 2/3 read
  double* t_dev;                   // stage 1 reads, stage 3 advances
  double* dt_user;                 // nullable copy of dt for the caller
  int nx, ny, bcx, bcy;
  int mask_mode;
  int stage;  // 0 = dU/dt; 1, 2, 3 = SSP-RK3 stages
  double dx, dy, gamma, gm1;
  double cfl, t_end;
  double third, two_thirds;
  double cand[4][4];   // candidate coefficients, stencil order
  double wtab[16][4];  // renormalised weights d_k / sum(kept d) per mask
  double teno[kTenoTable];  // TENO6-opt indicator matrices (mask_mode kMaskTeno)
};

struct RhsParamsF64 {
  RhsArgs a;
  NetF64 net;
};

struct ClassifyParamsF64 {
  const double* X;
  uint8_t* eta;
  double* logits;
  long long n;
  NetF64 net;
};

// Tensor-core image of the classifier (mixed precision): layers 1-4 as 16-bit
// B operands W_l[out][in] in the K-major canonical layout (K of layer 1
// padded to 16, N of layer 4 padded 8 -> 16 with zero rows).  In the bf16
// image layer 1's weights are split into two 16-bit terms, W1 = hi + lo
// (columns 0-5 hold hi, 6-11 lo), and the layer-1 input row carries the six
// stencil values in columns 0-5 and again in 6-11: the layer-1 products then
// see W1 to ~16 significant bits.  On smooth stencils the first layer's
// weights nearly cancel against the stencil's mean, and a single bf16
// rounding of W1 leaves a residue of the mean larger than the stencil's own
// variation.  The fp16 image keeps the single rounding and the plain row
// (stencil values in columns 0-5 only): at 11 bits the residue stays below
// the variation.  The biases of layers 1 and 2 ride on the tensor cores: the
// input row carries 1 in columns ones_col .. ones_col + 2 (6-8 in fp16, 12-14
// in bf16), B1 holds b1 split into
// three 16-bit terms (hi + mid + lo, ~24 significant bits) in those columns,
// and a fifth K-step of layer 2 multiplies the same input tile by the 32 x 16
// tile B2b that holds b2's three terms in those columns (zero elsewhere).  Then the FP32
// biases of layers 3-5 (b3 at 0, b4 at 16, b5 at 24) and the FP32 weights of
// layer 5, stored transposed (W5^T[8][4]) for packed two-output FMAs on the
// CUDA cores.
__host__ __device__ constexpr int ones_col(bool bf16) { return bf16 ? 12 : 6; }
constexpr int kNetImageB1 = 0;                           // 64 x 16
constexpr int kNetImageB2 = kNetImageB1 + 64 * 16 * 2;   // 32 x 64
constexpr int kNetImageB2b = kNetImageB2 + 32 * 64 * 2;  // 32 x 16
constexpr int kNetImageB3 = kNetImageB2b + 32 * 16 * 2;  // 16 x 32
constexpr int kNetImageB4 = kNetImageB3 + 16 * 32 * 2;   // 16 x 16
constexpr int kNetImageBias = kNetImageB4 + 16 * 16 * 2;
constexpr int kNetImageW5 = kNetImageBias + 32 * 4;
constexpr int kNetImageBytes = kNetImageW5 + 4 * 8 * 4;
static_assert(kNetImageBytes % 16 == 0, "image is copied in 16-byte chunks");

void build_net_image(const NetF64& net, bool bf16, uint8_t* img);

// The 6-32-32-32-4 network of the width study (neno6_classify only): its
// 2468 parameters occupy the start of NetF64 in the same packed order.  Its
// tensor-core image, in the same kNetImageBytes buffer: B1 32 x 16 (b1's
// terms in the ones columns), B2 32 x 32, B2b 32 x 16 (b2's terms), B3
// 32 x 32, then the FP32 b3[32], W4^T[32][4] and b4[4] (layer 4 on the CUDA
// cores).
constexpr int kNarrowWidths[5] = {6, 32, 32, 32, 4};
constexpr int kNarrowParams = 6 * 32 + 32 + 32 * 32 + 32 + 32 * 32 + 32 + 32 * 4 + 4;
static_assert(kNarrowParams == 2468 && kNarrowParams <= kNetParams, "6-32-32-32-4 parameter count");
constexpr int kNarrowB1 = 0;                          // 32 x 16
constexpr int kNarrowB2 = kNarrowB1 + 32 * 16 * 2;    // 32 x 32
constexpr int kNarrowB2b = kNarrowB2 + 32 * 32 * 2;   // 32 x 16
constexpr int kNarrowB3 = kNarrowB2b + 32 * 16 * 2;   // 32 x 32
constexpr int kNarrowBias3 = kNarrowB3 + 32 * 32 * 2;  // 32 floats
constexpr int kNarrowW4 = kNarrowBias3 + 32 * 4;       // 32 x 4 floats, then b4[4]
constexpr int kNarrowBytes = kNarrowW4 + 32 * 4 * 4 + 4 * 4;
static_assert(kNarrowBytes <= kNetImageBytes && kNarrowBytes % 16 == 0, "narrow image fits the buffer");
void build_net_image_narrow(const NetF64& net, bool bf16, uint8_t* img);
// FP32 parameters with every W transposed to [in][out] (guard re-evaluation).
void build_guard_image(const NetF64& net, float* img);

// Backward image of the classifier for the tensor-core gradient kernel: the
// transposed weights of layers 3 and 2 as 16-bit B operands (K-major, N x K
// = W3^T [32][16] and W2^T [64][32]), then W4 [8][16] and W5 [4][8] in FP32
// for the CUDA-core part of the backward pass.
constexpr int kBwdBW3 = 0;
constexpr int kBwdBW2 = kBwdBW3 + 32 * 16 * 2;
constexpr int kBwdW4 = kBwdBW2 + 64 * 32 * 2;
constexpr int kBwdW5 = kBwdW4 + 8 * 16 * 4;
constexpr int kBwdImageBytes = kBwdW5 + 4 * 8 * 4;
static_assert(kBwdImageBytes % 128 == 0, "backward image is copied in 16-byte chunks, 128-byte aligned");
void build_bwd_image(const NetF64& net, bool bf16, uint8_t* img);

// Linear weights d_k (printed optimal weights, or the sixth-order test
// weights), candidate coefficients of S0..S3 and the renormalised weights of
// every mask pattern: the tables every FP64 launch parameter block carries.
void scheme_tables(int linear_weights, double d[4], double cand[4][4], double wtab[16][4]);

// Mixed-precision face kernel arguments.
struct FacesMixedArgs {
  const double* U;
  double* Fx;  // [nv][ny][nx+1] x-face fluxes
  double* Fy;  // [nv][ny+1][nx] y-face fluxes
  uint8_t* mask_out;
  int* status;
  const uint8_t* net_image;  // tensor-core image
  const float* guard_w;      // FP32 transposed parameters
  unsigned long long* guard_count;
  int nx, ny, bcx, bcy;
  int mask_mode;
  int bf16;
  float guard_tau;
  double gamma, gm1;
  float cand[4][4];
  float wtab[16][4];
  // filled by the launcher: the launched x blocks are blk_x0 .. blk_x0 +
  // nblk_x - 1, then the y blocks blk_y0 .. blk_y0 + nblk_y - 1
  long long blk_x0, nblk_x, blk_y0, nblk_y;
  int bxf, byc;
};

struct DiffArgs {
  const double* Fx;
  const double* Fy;
  const double* U;   // stage input
  const double* U0;  // step start
  double* out;
  const double* dt_dev;
  double* t_dev;     // stage 3 advances *t_dev by dt (when not null)
  int nx, ny, stage;
  int bcx, bcy;
  int j0, j1;        // rows j0 .. j1 - 1
  double inv_dx, inv_dy, third, two_thirds;
};

// Face fluxes of the x faces of rows row0 .. row1 - 1 and of the y faces
// row0 .. row1 - 1 (.. ny when row1 == ny); row0 and row1 multiples of 16
// or row1 == ny.
cudaError_t launch_faces_mixed(int ndim, FacesMixedArgs& a, cudaStream_t s, int row0, int row1);
cudaError_t launch_diff_mixed(int ndim, const DiffArgs& a, cudaStream_t s);
// Wave-speed maxima of the cells of rows row0 .. row1 - 1 folded into smax
// (zeroed first when zero is set).
cudaError_t launch_cfl_mixed(int ndim, const double* U, int nx, int ny, double gamma, unsigned long long* smax,
                             int* status, cudaStream_t s, int row0, int row1, bool zero);
cudaError_t launch_dt(const unsigned long long* smax, int ndim, double dx, double dy, double cfl, double t_end,
                      const double* t_dev, double* dt_dev, double* dt_user, cudaStream_t s);

cudaError_t launch_rhs_fp64(int ndim, RhsParamsF64& p, cudaStream_t s);
cudaError_t launch_classify_mixed(const double* X, long long n, uint8_t* eta, double* logits,
                                  const uint8_t* net_image, bool bf16, bool narrow, int* status,
                                  cudaStream_t s);
cudaError_t launch_classify_fp64(const ClassifyParamsF64& p, bool narrow, cudaStream_t s);
// scratch: vjp_scratch_bytes(ndim, nx, ny) bytes (per-face contributions)
size_t vjp_scratch_bytes(int ndim, int nx, int ny);
cudaError_t launch_rhs_vjp(int ndim, const RhsArgs& a, const double* lam, double* grad, double* scratch,
                           cudaStream_t s);
int mlp_bwd_blocks(long long n);
size_t mlp_bwd_scratch_bytes(long long n);
cudaError_t launch_mlp_bwd(const double* X, const uint8_t* y, long long n, const float* params, float* grad,
                           float* loss, void* scratch, cudaStream_t s);
// The same gradient on the tensor cores (mixed-precision handles): 16-bit
// operands, FP32 accumulation; scratch of mlp_bwd_scratch_bytes(n) bytes.
cudaError_t launch_mlp_bwd_tc(const double* X, const uint8_t* y, long long n, const uint8_t* net_image,
                              const uint8_t* bwd_image, bool bf16, float* grad, float* loss, void* scratch,
                              int* status, cudaStream_t s);
// grad[p] = scale * (sum over the partial sums of the CTAs, in CTA order)
cudaError_t launch_mlp_bwd_reduce(const float* partial, const double* partial_loss, int blocks, long long n,
                                  float scale, float* grad, float* loss, cudaStream_t s);
// Scalar conservation laws (1D): law 0 linear advection, 1 Burgers.
struct ScalarParams {
  RhsArgs a;        // grid, boundary, mask mode, candidates, weights
  NetF64 net;
  int law;
  const double* u;  // [nx]
  double* F;        // [nx + 1] face fluxes
  uint8_t* mask_out;  // nullable [nx + 1]
};
cudaError_t launch_scalar_faces(const ScalarParams& p, cudaStream_t s);
cudaError_t launch_scalar_diff(const double* F, const double* in, const double* u0, double* out, int n,
                               double dx, int stage, double h, cudaStream_t s);
cudaError_t launch_scalar_speed(const double* u, int n, int law, unsigned long long* amax, cudaStream_t s);

// On-GPU classifier training: mini-batch Adam over a permutation of samples.
constexpr int kMaxTrainBatch = 192;
struct MlpTrainArgs {
  const double* X;     // [n][6] raw stencils
  const uint8_t* y;    // [n] label bits
  long long n;
  const int32_t* perm;  // [n_perm] sample indices, batches in this order
  long long n_perm;
  int batch;           // 1..kMaxTrainBatch; the last batch may be shorter
  float* params;       // [kNetParams] in/out
  float* m;            // [kNetParams] Adam first moments, in/out
  float* v;            // [kNetParams] Adam second moments, in/out
  long long t0;        // Adam steps taken before this call
  float lr;
  double* loss_sum;    // nullable: sum over the steps of the batch-mean loss
  int* status;
};
cudaError_t launch_mlp_train(const MlpTrainArgs& a, cudaStream_t s);
// Training data of Table 9 from uniform draws u [n][9] (csrc/datagen.cu).
cudaError_t launch_datagen(const double* u, long long n, double* X, uint8_t* labels, uint8_t* family,
                           int* status, cudaStream_t s);
cudaError_t launch_cfl_reduce(int ndim, const double* U, int nx, int ny, double gamma,
                              unsigned long long* smax, int* status, cudaStream_t s);

}  // namespace neno6
