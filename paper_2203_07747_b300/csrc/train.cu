// train.cu -- (a6) fitting the residual network to data (Sec. VI: MSE loss,
// Adam): the C ABI of the training calls and the drag-residual targets of
// the ground-truth simulator.  The training step itself (forward, loss,
// backward and weight-gradient GEMMs on the tensor cores, fused Adam) is in
// train_tc.cu.
#include <algorithm>
#include <cmath>
#include <string>

#include "rtn_internal.cuh"

namespace rtn {
namespace {

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

// training buffers for minibatches of up to cap samples, planned for bs
rtn_status ensure_train(rtn_ctx* ctx, int cap, int bs) {
  std::string e;
  cudaError_t ce = train_prepare(ctx, ctx->train, std::max(cap, ctx->train.cap), bs, e);
  if (ce != cudaSuccess)
    return tfail(ctx, ce == cudaErrorMemoryAllocation ? RTN_E_NOMEM : RTN_E_CUDA,
                 std::string("training buffers: ") + cudaGetErrorString(ce));
  if (!e.empty()) return tfail(ctx, RTN_E_CUDA, e);
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
  if (ctx->opt.precision == RTN_FP8) {
    // the trained master weights quantised again (e4m3, scale amax/448)
    for (int l = 0; l < L; ++l)
      net.fp8_scale[l] = quantize_e4m3(W.data() + net.w_off[l], (size_t)net.widths[l + 1] * net.widths[l]);
    TCK(cudaMemcpy(net.W32, W.data(), ts.nw * 4, cudaMemcpyHostToDevice));
    // the split copies the training GEMMs use follow the quantised weights
    TCK(train_resplit(ctx, ts));
  }
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
  rtn_status st = ensure_train(ctx, n, n);
  if (st != RTN_OK) return st;
  TrainState& ts = ctx->train;
  TCK(cudaMemsetAsync(loss, 0, sizeof(float), ctx->stream));
  TCK(train_grad(ctx, ts, X, U, Y, 0, loss));
  TCK(train_reduce(ctx, ts));
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
  rtn_status st = ensure_train(ctx, batch, batch);
  if (st != RTN_OK) return st;
  TrainState& ts = ctx->train;
  const int per_epoch = n / batch;
  const long long steps = (long long)epochs * per_epoch;
  float* dloss = nullptr;
  TCK(cudaMalloc(&dloss, std::max<long long>(steps, 1) * sizeof(float)));
  TCK(cudaMemsetAsync(dloss, 0, std::max<long long>(steps, 1) * sizeof(float), ctx->stream));
  cudaError_t e = cudaSuccess;
  // one training step (~5 L launches) captured as a CUDA graph on a stream of
  // its own and replayed `steps` times: the minibatch and the loss entry come
  // from a step counter on the device that the step advances at its end, and
  // the Adam step counter lives on the device too
  cudaStream_t user = ctx->stream, cs = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev = nullptr;
  int* k_dev = nullptr;
  if (steps > 0) {
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&k_dev, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(k_dev, 0, sizeof(int), user);
    if (e == cudaSuccess) e = cudaEventRecord(ev, user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev, 0);
    if (e == cudaSuccess) {
      ctx->stream = cs;
      e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        e = train_grad_dev(ctx, ts, X, U, Y, k_dev, per_epoch, dloss);
        if (e == cudaSuccess) e = train_adam(ctx, ts, lr, k_dev);
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = e2;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
      ts.t -= 1;  // train_adam advanced the host mirror while recording
    }
    for (long long k = 0; k < steps && e == cudaSuccess; ++k) {
      e = cudaGraphLaunch(exec, cs);
      ts.t += 1;
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev, cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(user, ev, 0);
    ctx->stream = user;
  }
  if (e == cudaSuccess && loss_out && steps > 0)
    e = cudaMemcpyAsync(loss_out, dloss, steps * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = ctx->stream ? cudaStreamSynchronize(ctx->stream) : cudaDeviceSynchronize();
  if (cs) cudaStreamSynchronize(cs);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (ev) cudaEventDestroy(ev);
  if (cs) cudaStreamDestroy(cs);
  if (k_dev) cudaFree(k_dev);
  cudaFree(dloss);
  ctx->stream = user;
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
