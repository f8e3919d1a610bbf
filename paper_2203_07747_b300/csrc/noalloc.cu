// noalloc.cu -- FP32 network value + Jacobian for callers that cannot
// allocate device memory.
//
// rtn_mlp_eval needs a context from rtn_create, which allocates the
// activation buffers of the FP32 path with cudaMalloc.  Some callers cannot
// do that: hosts that hand out all device memory themselves (a fixed pool or
// a certified real-time runtime where dynamic allocation after start-up is
// forbidden, because cudaMalloc may synchronise the device and has no bounded
// latency).  rtn_mlp_eval_f32_noalloc runs the same FP32 kernels with their
// activations in a fixed array compiled into the library, so it calls no
// allocator at all.  The paper has no counterpart of this entry point.
//
// The array is RTN_NOALLOC_SCRATCH_BYTES large on every GPU that loads the
// library and stays there until the process exits.  All calls share it: two
// calls whose kernels overlap on the GPU (different streams, other threads)
// race on it.  Its previous contents never matter: every element a kernel
// reads was written earlier in the same call.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>
#include <string>

#include "rtn_internal.cuh"

namespace {

using namespace rtn;

constexpr size_t kScratchFloats = RTN_NOALLOC_SCRATCH_BYTES / sizeof(float);
static __device__ __align__(256) float g_noalloc_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
// per device: the array's device address and the context it was looked up
// in (a device reset makes a new primary context; the address is looked up
// again there)
float* g_scratch_ptr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};

// the calling thread's current driver context (null if none or unavailable)
CUcontext current_context() {
  static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
  static bool looked = false;
  if (!looked) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &qr) == cudaSuccess &&
        qr == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
    looked = true;
  }
  CUcontext c = nullptr;
  if (fn) fn(&c);
  return c;
}

// input layer for nodes given as separate rows x[n][13], u[n][4]: one thread
// per (neuron i, node n, column c) with c fastest, so that a warp stores
// consecutive floats of the [h0][18 n_nodes] block (each thread recomputes
// its node's 17-term dot product)
__global__ void noalloc_in_kernel(const float* __restrict__ x, const float* __restrict__ u,
                                  int n_nodes, const float* __restrict__ W0,
                                  const float* __restrict__ b0, int h0, float* __restrict__ X1) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per_row = (long long)NC * n_nodes;
  if (tid >= (long long)h0 * per_row) return;
  const int i = (int)(tid / per_row);
  const long long r = tid % per_row;
  const int n = (int)(r / NC), c = (int)(r % NC);
  const float* xr = x + (size_t)n * NX;
  const float* ur = u + (size_t)n * NU;
  const float* w = W0 + (size_t)i * NZ;
  float s = b0[i];
#pragma unroll
  for (int j = 0; j < NX; ++j) s = fmaf(w[j], xr[j], s);
#pragma unroll
  for (int j = 0; j < NU; ++j) s = fmaf(w[NX + j], ur[j], s);
  const float a = tanhf(s);
  X1[(size_t)i * per_row + r] = c == 0 ? a : (1.0f - a * a) * w[c - 1];
}

rtn_status fail(char* err, size_t len, rtn_status st, const std::string& msg) {
  if (err && len) {
    size_t n = msg.size() < len - 1 ? msg.size() : len - 1;
    msg.copy(err, n);
    err[n] = '\0';
  }
  return st;
}

}  // namespace

extern "C" rtn_status rtn_mlp_eval_f32_noalloc(int n_layers, const int* widths, const float* W,
                                               const float* b, int n_nodes, const float* x,
                                               const float* u, float* fD, float* JD,
                                               void* cuda_stream, char* err, size_t err_len) {
  if (err && err_len) err[0] = '\0';
  if (n_layers < 2 || !widths || widths[0] != NZ || widths[n_layers] != NO)
    return fail(err, err_len, RTN_E_INVAL, "network must map 17 inputs to 3 outputs");
  if (!W || !b || !x || !u || !fD || !JD || n_nodes < 1)
    return fail(err, err_len, RTN_E_INVAL, "NULL pointer or n_nodes < 1");
  long long h_max = 0;
  for (int l = 1; l < n_layers; ++l) {
    if (widths[l] < 1) return fail(err, err_len, RTN_E_INVAL, "hidden width < 1");
    if (widths[l] > h_max) h_max = widths[l];
  }
  const long long need = 2LL * h_max * NC * n_nodes;  // two activation buffers
  if (need > (long long)kScratchFloats)
    return fail(err, err_len, RTN_E_INVAL,
                "needs " + std::to_string(need * 4) + " bytes of activation scratch; the static "
                "buffer holds " + std::to_string((long long)RTN_NOALLOC_SCRATCH_BYTES) +
                " (reduce n_nodes or the hidden width)");

  // once per device (and again after a device reset), with that device
  // current: the device address of the array
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(err, err_len, RTN_E_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(err, err_len, RTN_E_UNSUPPORTED, "device index");
  float* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    const CUcontext cur = current_context();
    if (!g_scratch_ptr[dev] || (cur && cur != g_scratch_ctx[dev])) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess)
        return fail(err, err_len, RTN_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_ptr[dev] = static_cast<float*>(p);
      g_scratch_ctx[dev] = current_context();
    }
    scratch = g_scratch_ptr[dev];
  }

  cudaStream_t s = (cudaStream_t)cuda_stream;
  float* cur = scratch;
  float* nxt = scratch + (size_t)h_max * NC * n_nodes;
  size_t wo = 0, bo = 0;
  {
    int h0 = widths[1];
    long long tot = (long long)h0 * NC * n_nodes;
    noalloc_in_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(x, u, n_nodes, W, b, h0, cur);
    e = cudaGetLastError();
    wo += (size_t)h0 * NZ;
    bo += h0;
  }
  for (int l = 1; l < n_layers - 1 && e == cudaSuccess; ++l) {
    int K = widths[l], M = widths[l + 1];
    e = mlp_f32_hidden_launch(W + wo, b + bo, M, K, cur, nxt, n_nodes, s);
    wo += (size_t)M * K;
    bo += M;
    float* t = cur; cur = nxt; nxt = t;
  }
  if (e == cudaSuccess)
    e = mlp_f32_out_launch(W + wo, b + bo, widths[n_layers - 1], cur, n_nodes, fD, JD, s);
  if (e != cudaSuccess) return fail(err, err_len, RTN_E_CUDA, cudaGetErrorString(e));
  return RTN_OK;
}
