// mlp_f32.cu -- (a1) residual network value + input Jacobian, FP32 SIMT
// kernels of the allocation-free entry point (noalloc.cu; controller contexts
// evaluate the network on the tensor cores, mlp_tf32.cu).
//
// Forward-mode differentiation of f_D (Sec. III-A, Eq. 4): every node carries
// 18 columns through the network, its value and the 17 tangent directions
// d/d[x;u].  With the activations of all nodes stored as one matrix
// X_l [h_l][18 n_nodes] (column 18 n + j = node n, column j), a hidden layer
// is one GEMM  Z = W_l X_l  followed by an epilogue that, per node and
// neuron, takes the value column a = tanh(z + b) and scales the 17 tangent
// columns by tanh' = 1 - a^2.  The input layer needs no GEMM (its tangent is
// W_0 itself) and the 3-row output layer is a thin reduction.
#include "rtn_internal.cuh"

namespace rtn {
namespace {

// hidden layer GEMM with the fused tanh / tanh' epilogue.
// Tile: 128 neurons x 8 nodes (144 columns), K in slices of 16.  Thread
// (rg, ng): rows 8 rg .. 8 rg + 7 of the tile, node ng -> 8 x 18 accumulators,
// so the whole value/tangent block of a node is in one thread's registers.
constexpr int BM = 128, BNN = 8, BN = BNN * NC, BK = 16, NTH = 128;

__global__ void __launch_bounds__(NTH) mlp_hidden_kernel(const float* __restrict__ W,
                                                         const float* __restrict__ bias, int M,
                                                         int K, const float* __restrict__ X,
                                                         float* __restrict__ Y, int n_nodes) {
  __shared__ __align__(16) float As[BK][BM];
  __shared__ __align__(16) float Bs[BK][BN];
  const size_t ldx = (size_t)NC * n_nodes;
  const int tid = threadIdx.x, rg = tid & 15, ng = tid >> 4;
  const int m0 = blockIdx.y * BM;
  const int node0 = blockIdx.x * BNN;
  const size_t col0 = (size_t)node0 * NC;
  const int ncols = (int)min((size_t)BN, ldx - col0);
  float acc[8][NC];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int j = 0; j < NC; ++j) acc[r][j] = 0.0f;

  for (int k0 = 0; k0 < K; k0 += BK) {
    {
      int m = m0 + tid;
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        int k = k0 + kk;
        As[kk][tid] = (m < M && k < K) ? W[(size_t)m * K + k] : 0.0f;
      }
    }
#pragma unroll
    for (int it = 0; it < (BK * BN) / NTH; ++it) {
      int e = it * NTH + tid;
      int kk = e / BN, cc = e % BN;
      int k = k0 + kk;
      Bs[kk][cc] = (k < K && cc < ncols) ? X[(size_t)k * ldx + col0 + cc] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[8], b[NC];
      const float4* ap = reinterpret_cast<const float4*>(&As[kk][rg * 8]);
      float4 a0 = ap[0], a1 = ap[1];
      a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
      a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
      const float2* bp = reinterpret_cast<const float2*>(&Bs[kk][ng * NC]);
#pragma unroll
      for (int j = 0; j < NC / 2; ++j) {
        float2 t = bp[j];
        b[2 * j] = t.x; b[2 * j + 1] = t.y;
      }
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int j = 0; j < NC; ++j) acc[r][j] = fmaf(a[r], b[j], acc[r][j]);
    }
    __syncthreads();
  }
  int node = node0 + ng;
  if (node >= n_nodes) return;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    int m = m0 + rg * 8 + r;
    if (m >= M) continue;
    float av = tanhf(acc[r][0] + bias[m]);
    float d = 1.0f - av * av;
    float2* o = reinterpret_cast<float2*>(Y + (size_t)m * ldx + (size_t)node * NC);
    o[0] = make_float2(av, acc[r][1] * d);
#pragma unroll
    for (int j = 1; j < NC / 2; ++j) o[j] = make_float2(acc[r][2 * j] * d, acc[r][2 * j + 1] * d);
  }
}

// output layer (NOUT rows, linear: 3, or 6 for the full residual):
// thread (node n, column j) computes the outputs of its column
template <int NOUT>
__global__ void mlp_out_kernel(const float* __restrict__ WL, const float* __restrict__ bL, int K,
                               const float* __restrict__ X, int n_nodes, float* __restrict__ fD,
                               float* __restrict__ JD) {
  long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (long long)n_nodes * NC) return;
  int n = (int)(tid / NC), j = (int)(tid % NC);
  const size_t ldx = (size_t)NC * n_nodes;
  const float* xc = X + (size_t)n * NC + j;
  float s[NOUT];
#pragma unroll
  for (int r = 0; r < NOUT; ++r) s[r] = 0.f;
  for (int k = 0; k < K; ++k) {
    float v = xc[(size_t)k * ldx];
#pragma unroll
    for (int r = 0; r < NOUT; ++r) s[r] = fmaf(WL[r * K + k], v, s[r]);
  }
  if (j == 0) {
#pragma unroll
    for (int r = 0; r < NOUT; ++r) fD[(size_t)n * NOUT + r] = s[r] + bL[r];
  } else {
    float* o = JD + (size_t)n * NOUT * NZ + (j - 1);
#pragma unroll
    for (int r = 0; r < NOUT; ++r) o[r * NZ] = s[r];
  }
}

}  // namespace

cudaError_t mlp_f32_hidden_launch(const float* W, const float* bias, int M, int K, const float* X,
                                  float* Y, int n_nodes, cudaStream_t s) {
  dim3 grid((n_nodes + BNN - 1) / BNN, (M + BM - 1) / BM);
  mlp_hidden_kernel<<<grid, NTH, 0, s>>>(W, bias, M, K, X, Y, n_nodes);
  return cudaGetLastError();
}

cudaError_t mlp_f32_out_launch(const float* WL, const float* bL, int K, const float* X,
                               int n_nodes, float* fD, float* JD, cudaStream_t s) {
  long long tot = (long long)n_nodes * NC;
  mlp_out_kernel<NO><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(WL, bL, K, X, n_nodes, fD, JD);
  return cudaGetLastError();
}

}  // namespace rtn
