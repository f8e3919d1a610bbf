// train.cu -- (a6) fitting the residual network to data (Sec. VI: MSE loss,
// Adam), plus the drag-residual targets of the ground-truth simulator.
//
// A training step on a minibatch of `bs` samples, activations feature-major
// (A_l is [h_l][bs], batch contiguous):
//   forward   Z_l = W_l A_{l-1} + b_l,  A_l = tanh(Z_l) (hidden), A_L = Z_L
//   loss      L = 1/(3 bs) sum (A_L - Y)^2,  G_L = 2 (A_L - Y) / (3 bs)
//   backward  dW_l = G_l A_{l-1}',  db_l = sum_batch G_l,
//             G_{l-1} = (W_l' G_l) * (1 - A_{l-1}^2)
//   Adam      one fused launch over all parameters (FP32 master weights).
// The GEMMs run in cuBLAS (FP32 emulated on the tensor cores), the rest in
// the kernels below.
#include <algorithm>
#include <cmath>
#include <string>

#include <cublas_v2.h>

#include "rtn_internal.cuh"

namespace rtn {
namespace {

// C[M][N] (row-major, ldc) = op(A)[M][K] op(B)[K][N]
// op(A)(m,k) = TA ? A[k*lda + m] : A[m*lda + k];  op(B)(k,n) = TB ? B[n*ldb + k] : B[k*ldb + n]
// These are plain GEMMs (the bias, activation and loss epilogues are kernels
// of their own), so they run in cuBLAS on the tensor cores with FP32
// emulated by BF16 splits (CUBLAS_COMPUTE_32F_EMULATED_16BFX9, FP32-level
// accuracy).  Row-major C = op(A) op(B) is column-major C' = op(B)' op(A)'.
template <bool TA, bool TB>
cudaError_t sgemm(TrainState& ts, int M, int N, int K, const float* A, int lda, const float* B, int ldb,
                  float* C, int ldc, cudaStream_t s) {
  cublasHandle_t h = static_cast<cublasHandle_t>(ts.blas);
  const float one = 1.0f, zero = 0.0f;
  cublasStatus_t st = cublasSetStream(h, s);
  if (st == CUBLAS_STATUS_SUCCESS)
    st = cublasGemmEx(h, TB ? CUBLAS_OP_T : CUBLAS_OP_N, TA ? CUBLAS_OP_T : CUBLAS_OP_N, N, M, K, &one, B,
                      CUDA_R_32F, ldb, A, CUDA_R_32F, lda, &zero, C, CUDA_R_32F, ldc,
                      CUBLAS_COMPUTE_32F_EMULATED_16BFX9, CUBLAS_GEMM_DEFAULT);
  if (st == CUBLAS_STATUS_SUCCESS) return cudaSuccess;
  return st == CUBLAS_STATUS_NOT_SUPPORTED ? cudaErrorNotSupported : cudaErrorUnknown;
}

// A_0 [17][bs] from samples [start, start + bs) of X [n][13], U [n][4]
__global__ void gather_input_kernel(const float* __restrict__ X, const float* __restrict__ U,
                                    int start, int bs, float* __restrict__ A0) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NZ * bs) return;
  int j = i / bs, s = i % bs;
  size_t r = (size_t)start + s;
  A0[i] = j < NX ? X[r * NX + j] : U[r * NU + (j - NX)];
}

// Z += b (per row), then tanh unless linear
__global__ void bias_act_kernel(float* __restrict__ Z, const float* __restrict__ b, int rows, int bs,
                                int linear) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * bs) return;
  float v = Z[i] + b[i / bs];
  Z[i] = linear ? v : tanhf(v);
}

// G = 2 (Yhat - Y) / (no bs), loss partial sums (one atomicAdd per block);
// no = the network's outputs (3, or 6 for the full residual)
__global__ void loss_grad_kernel(const float* __restrict__ Yh, const float* __restrict__ Y, int start,
                                 int bs, int no, float* __restrict__ G, float* __restrict__ loss) {
  __shared__ float red[256];
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  float e2 = 0.0f;
  if (i < no * bs) {
    int r = i / bs, s = i % bs;
    float e = Yh[i] - Y[((size_t)start + s) * no + r];
    G[i] = 2.0f * e / ((float)no * bs);
    e2 = e * e;
  }
  red[threadIdx.x] = e2;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0] / ((float)no * bs));
}

// db[r] = sum over the batch of G[r][:]  (one block per row)
__global__ void rowsum_kernel(const float* __restrict__ G, int bs, float* __restrict__ db) {
  __shared__ float red[256];
  float s = 0.0f;
  for (int i = threadIdx.x; i < bs; i += 256) s += G[(size_t)blockIdx.x * bs + i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[blockIdx.x] = red[0];
}

// G *= 1 - A^2 (tanh' from the stored activation)
__global__ void tanh_back_kernel(float* __restrict__ G, const float* __restrict__ A, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) G[i] *= 1.0f - A[i] * A[i];
}

// fused Adam over all parameters, bias-corrected, step t >= 1
__global__ void adam_kernel(float* __restrict__ P, const float* __restrict__ Gp, float* __restrict__ m,
                            float* __restrict__ v, size_t n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float g = Gp[i];
  float mi = b1 * m[i] + (1.0f - b1) * g;
  float vi = b2 * v[i] + (1.0f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// drag residual of the ground-truth simulator, per sample (FP32):
// a = -R(q) diag(0.3, 0.3, 0.1) R(q)' v - 0.01 |v| v
__global__ void drag_kernel(const float* __restrict__ X, int n, float* __restrict__ Y) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const float* x = X + (size_t)s * NX;
  float qw = x[3], qx = x[4], qy = x[5], qz = x[6], vx = x[7], vy = x[8], vz = x[9];
  // rotation matrix of q (literal q v q^* for unit q)
  float R[3][3] = {{qw * qw + qx * qx - qy * qy - qz * qz, 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy)},
                   {2 * (qx * qy + qw * qz), qw * qw - qx * qx + qy * qy - qz * qz, 2 * (qy * qz - qw * qx)},
                   {2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), qw * qw - qx * qx - qy * qy + qz * qz}};
  float vb[3], db[3];
  for (int i = 0; i < 3; ++i) vb[i] = R[0][i] * vx + R[1][i] * vy + R[2][i] * vz;
  db[0] = 0.3f * vb[0]; db[1] = 0.3f * vb[1]; db[2] = 0.1f * vb[2];
  float nv = sqrtf(vx * vx + vy * vy + vz * vz);
  float v[3] = {vx, vy, vz};
  for (int i = 0; i < 3; ++i)
    Y[(size_t)s * NO + i] = -(R[i][0] * db[0] + R[i][1] * db[1] + R[i][2] * db[2]) - 0.01f * nv * v[i];
}

inline unsigned blocks(size_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t drag_targets(rtn_ctx* ctx, const float* X, int n, float* Y) {
  drag_kernel<<<blocks(n), 256, 0, ctx->stream>>>(X, n, Y);
  return cudaGetLastError();
}

// loss and gradient of one minibatch into ts.grad; `loss` (device scalar)
// is accumulated
cudaError_t train_grad(rtn_ctx* ctx, TrainState& ts, const float* X, const float* U, const float* Y,
                       int start, float* loss) {
  Net& net = ctx->net;
  const int L = net.n_layers, bs = ts.bs;
  cudaStream_t s = ctx->stream;
  // forward
  gather_input_kernel<<<blocks((size_t)NZ * bs), 256, 0, s>>>(X, U, start, bs, ts.act[0]);
  for (int l = 0; l < L; ++l) {
    const int fi = net.widths[l], fo = net.widths[l + 1];
    cudaError_t e = sgemm<false, false>(ts, fo, bs, fi, net.W32 + net.w_off[l], fi, ts.act[l], bs, ts.act[l + 1],
                                        bs, s);
    if (e != cudaSuccess) return e;
    bias_act_kernel<<<blocks((size_t)fo * bs), 256, 0, s>>>(ts.act[l + 1], net.b32 + net.b_off[l], fo,
                                                            bs, l == L - 1);
  }
  const int no = net.widths[L];
  loss_grad_kernel<<<blocks((size_t)no * bs), 256, 0, s>>>(ts.act[L], Y, start, bs, no, ts.g0, loss);
  // backward
  float* G = ts.g0;
  float* Gn = ts.g1;
  for (int l = L - 1; l >= 0; --l) {
    const int fi = net.widths[l], fo = net.widths[l + 1];
    cudaError_t e = sgemm<false, true>(ts, fo, fi, bs, G, bs, ts.act[l], bs, ts.grad + net.w_off[l], fi, s);
    if (e != cudaSuccess) return e;
    rowsum_kernel<<<fo, 256, 0, s>>>(G, bs, ts.grad + ts.b_base + net.b_off[l]);
    if (l > 0) {
      e = sgemm<true, false>(ts, fi, bs, fo, net.W32 + net.w_off[l], fi, G, bs, Gn, bs, s);
      if (e != cudaSuccess) return e;
      tanh_back_kernel<<<blocks((size_t)fi * bs), 256, 0, s>>>(Gn, ts.act[l], fi * bs);
      float* t = G; G = Gn; Gn = t;
    }
  }
  return cudaGetLastError();
}

// one minibatch step: gradient, then Adam on weights and biases
cudaError_t train_step(rtn_ctx* ctx, TrainState& ts, const float* X, const float* U, const float* Y,
                       int start, float lr, float* loss) {
  Net& net = ctx->net;
  cudaStream_t s = ctx->stream;
  cudaError_t e = train_grad(ctx, ts, X, U, Y, start, loss);
  if (e != cudaSuccess) return e;
  ts.t += 1;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.0f - powf(b1, (float)ts.t), c2 = 1.0f - powf(b2, (float)ts.t);
  adam_kernel<<<blocks(ts.nw), 256, 0, s>>>(net.W32, ts.grad, ts.m, ts.v, ts.nw, lr, b1, b2, eps, c1, c2);
  adam_kernel<<<blocks(ts.nb), 256, 0, s>>>(net.b32, ts.grad + ts.b_base, ts.m + ts.nw, ts.v + ts.nw, ts.nb,
                                            lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

}  // namespace rtn

// ------------------------------------------------------------------ C ABI

namespace {

using namespace rtn;

rtn_status tfail(rtn_ctx* ctx, rtn_status st, const std::string& m) {
  ctx->err = m;
  return st;
}

#define TCK(call)                                                              \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) return tfail(ctx, e_ == cudaErrorMemoryAllocation ? RTN_E_NOMEM : RTN_E_CUDA, \
                                        std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// (re)allocate the training buffers for minibatches of bs samples
rtn_status ensure_train(rtn_ctx* ctx, int bs) {
  TrainState& ts = ctx->train;
  Net& net = ctx->net;
  const int L = net.n_layers;
  if (!ts.blas) {
    cublasHandle_t h = nullptr;
    if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) return tfail(ctx, RTN_E_CUDA, "cublasCreate failed");
    ts.blas = h;
    // emulate FP32 on the tensor cores for every size (not only where the
    // library expects a gain)
    if (cublasSetEmulationStrategy(h, CUBLAS_EMULATION_STRATEGY_EAGER) != CUBLAS_STATUS_SUCCESS)
      return tfail(ctx, RTN_E_CUDA, "cublasSetEmulationStrategy failed");
  }
  if (!ts.grad) {
    ts.nw = 0;
    ts.nb = 0;
    for (int l = 0; l < L; ++l) {
      ts.nw += (size_t)net.widths[l + 1] * net.widths[l];
      ts.nb += net.widths[l + 1];
    }
    ts.b_base = ts.nw;
    TCK(cudaMalloc(&ts.grad, (ts.nw + ts.nb) * sizeof(float)));
    TCK(cudaMalloc(&ts.m, (ts.nw + ts.nb) * sizeof(float)));
    TCK(cudaMalloc(&ts.v, (ts.nw + ts.nb) * sizeof(float)));
    TCK(cudaMemset(ts.m, 0, (ts.nw + ts.nb) * sizeof(float)));
    TCK(cudaMemset(ts.v, 0, (ts.nw + ts.nb) * sizeof(float)));
    ts.t = 0;
  }
  if (ts.bs < bs) {
    for (float* p : ts.act) cudaFree(p);
    ts.act.clear();
    if (ts.g0) cudaFree(ts.g0);
    if (ts.g1) cudaFree(ts.g1);
    ts.g0 = ts.g1 = nullptr;
    ts.act.assign(L + 1, nullptr);
    int hmax = 0;
    for (int l = 0; l <= L; ++l) {
      hmax = std::max(hmax, net.widths[l]);
      TCK(cudaMalloc(&ts.act[l], (size_t)net.widths[l] * bs * sizeof(float)));
    }
    TCK(cudaMalloc(&ts.g0, (size_t)hmax * bs * sizeof(float)));
    TCK(cudaMalloc(&ts.g1, (size_t)hmax * bs * sizeof(float)));
    ts.bs = bs;
  }
  return RTN_OK;
}

// after the FP32 master weights changed: FP64 plant copy and the tensor-core
// packs (split BF16, or the TF32 hi/lo weights of RTN_FP32 contexts)
rtn_status refresh_network(rtn_ctx* ctx) {
  Net& net = ctx->net;
  const int L = net.n_layers;
  TrainState& ts = ctx->train;
  std::vector<float> W(ts.nw), b(ts.nb);
  TCK(cudaStreamSynchronize(ctx->stream));
  TCK(cudaMemcpy(W.data(), net.W32, ts.nw * 4, cudaMemcpyDeviceToHost));
  TCK(cudaMemcpy(b.data(), net.b32, ts.nb * 4, cudaMemcpyDeviceToHost));
  std::vector<double> P;
  for (int l = 0; l < L; ++l) {
    const size_t nwl = (size_t)net.widths[l + 1] * net.widths[l];
    P.insert(P.end(), W.begin() + net.w_off[l], W.begin() + net.w_off[l] + nwl);
    P.insert(P.end(), b.begin() + net.b_off[l], b.begin() + net.b_off[l] + net.widths[l + 1]);
  }
  TCK(cudaMemcpy(net.P64, P.data(), P.size() * sizeof(double), cudaMemcpyHostToDevice));
  if (ctx->opt.precision != RTN_FP32) {
    const int keep = net.tc.variant;
    mlp_tc_release(ctx);
    std::string e;
    cudaError_t ce = mlp_tc_prepare(ctx, e);
    if (ce != cudaSuccess || !e.empty()) return tfail(ctx, RTN_E_CUDA, "repacking the network: " + e);
    if (keep >= 0 && mlp_tc_variant_info(ctx, keep, nullptr, nullptr, nullptr) == 0)
      TCK(mlp_tc_select(ctx, keep));
  } else if (ctx->tf) {
    const int mode = ctx->tf->mode;
    mlp_tf32_release(ctx);
    std::string e;
    cudaError_t ce = mlp_tf32_prepare(ctx, mode, e);
    if (ce != cudaSuccess || !e.empty()) return tfail(ctx, RTN_E_CUDA, "repacking the network: " + e);
  }
  return RTN_OK;
}

}  // namespace

extern "C" {

rtn_status rtn_drag_targets(rtn_ctx* ctx, const float* X, int n, float* Y) {
  if (!ctx) return RTN_E_INVAL;
  if (ctx->di) {
    ctx->err = "rtn_drag_targets: not available for the double-integrator model";
    return RTN_E_UNSUPPORTED;
  }
  if (!X || !Y || n < 1) return tfail(ctx, RTN_E_INVAL, "rtn_drag_targets: bad argument");
  TCK(drag_targets(ctx, X, n, Y));
  return RTN_OK;
}

rtn_status rtn_mse_grad(rtn_ctx* ctx, const float* X, const float* U, const float* Y, int n,
                        float* grad, float* loss) {
  if (!ctx) return RTN_E_INVAL;
  if (ctx->di) {
    ctx->err = "rtn_mse_grad: not available for the double-integrator model";
    return RTN_E_UNSUPPORTED;
  }
  if (!ctx->has_mlp) return tfail(ctx, RTN_E_UNSUPPORTED, "rtn_mse_grad: no network");
  if (!X || !U || !Y || n < 1 || !grad || !loss) return tfail(ctx, RTN_E_INVAL, "rtn_mse_grad: bad argument");
  rtn_status st = ensure_train(ctx, n);
  if (st != RTN_OK) return st;
  TrainState& ts = ctx->train;
  TCK(cudaMemsetAsync(loss, 0, sizeof(float), ctx->stream));
  // the buffers are sized for ts.bs >= n; run on exactly n samples
  const int keep = ts.bs;
  ts.bs = n;
  cudaError_t e = train_grad(ctx, ts, X, U, Y, 0, loss);
  ts.bs = keep;
  TCK(e);
  TCK(cudaMemcpyAsync(grad, ts.grad, (ts.nw + ts.nb) * sizeof(float), cudaMemcpyDeviceToDevice,
                      ctx->stream));
  return RTN_OK;
}

rtn_status rtn_train(rtn_ctx* ctx, const float* X, const float* U, const float* Y, int n,
                     int epochs, int batch, float lr, float* loss_out) {
  if (!ctx) return RTN_E_INVAL;
  if (ctx->di) {
    ctx->err = "rtn_train: not available for the double-integrator model";
    return RTN_E_UNSUPPORTED;
  }
  if (!ctx->has_mlp) return tfail(ctx, RTN_E_UNSUPPORTED, "rtn_train: no network");
  if (!X || !U || !Y || n < 1 || epochs < 0 || batch < 1 || batch > n || !(lr > 0.0f))
    return tfail(ctx, RTN_E_INVAL, "rtn_train: bad argument");
  rtn_status st = ensure_train(ctx, batch);
  if (st != RTN_OK) return st;
  TrainState& ts = ctx->train;
  const int keep = ts.bs;
  ts.bs = batch;
  const int per_epoch = n / batch;
  const long long steps = (long long)epochs * per_epoch;
  float* dloss = nullptr;
  TCK(cudaMalloc(&dloss, std::max<long long>(steps, 1) * sizeof(float)));
  TCK(cudaMemsetAsync(dloss, 0, std::max<long long>(steps, 1) * sizeof(float), ctx->stream));
  cudaError_t e = cudaSuccess;
  for (long long k = 0; k < steps && e == cudaSuccess; ++k)
    e = train_step(ctx, ts, X, U, Y, (int)(k % per_epoch) * batch, lr, dloss + k);
  ts.bs = keep;
  if (e == cudaSuccess && loss_out && steps > 0)
    e = cudaMemcpyAsync(loss_out, dloss, steps * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(dloss);
  TCK(e);
  return refresh_network(ctx);
}

rtn_status rtn_get_params(rtn_ctx* ctx, float* W, float* b) {
  if (!ctx) return RTN_E_INVAL;
  if (ctx->di) {
    ctx->err = "rtn_get_params: not available for the double-integrator model";
    return RTN_E_UNSUPPORTED;
  }
  if (!ctx->has_mlp || !W || !b) return tfail(ctx, RTN_E_INVAL, "rtn_get_params: bad argument");
  size_t nw = 0, nb = 0;
  for (int l = 0; l < ctx->net.n_layers; ++l) {
    nw += (size_t)ctx->net.widths[l + 1] * ctx->net.widths[l];
    nb += ctx->net.widths[l + 1];
  }
  TCK(cudaStreamSynchronize(ctx->stream));
  TCK(cudaMemcpy(W, ctx->net.W32, nw * 4, cudaMemcpyDeviceToHost));
  TCK(cudaMemcpy(b, ctx->net.b32, nb * 4, cudaMemcpyDeviceToHost));
  return RTN_OK;
}

}  // extern "C"

namespace rtn {
void train_release(rtn_ctx* ctx) {
  TrainState& ts = ctx->train;
  for (float* p : ts.act) if (p) cudaFree(p);
  void* ptrs[] = {ts.g0, ts.g1, ts.grad, ts.m, ts.v};
  for (void* p : ptrs) if (p) cudaFree(p);
  if (ts.blas) cublasDestroy(static_cast<cublasHandle_t>(ts.blas));
  ts = TrainState{};
}
}  // namespace rtn
