// mlp_hess.cu -- the second-order local model of Eq. 4: f_D, J_D and the
// Hessian H_D of the residual network at every node (FP32 SIMT).
//
// Forward-over-forward differentiation: every node carries 171 columns
// through the network -- the value, the 17 tangents t_j = da/dz_j and the 153
// second derivatives s_jm = d^2 a / dz_j dz_m (j <= m).  With the layout of
// the FP32 path (X_l [h_l][171 n_nodes], node-major column blocks), a hidden
// layer is a plain GEMM Z = W_l X_l (h2_gemm_kernel) followed by an
// elementwise kernel (h2_act_kernel) that forms, per neuron and node,
//   a = tanh(z_0 + b),  t_j = tanh'(.) z_j,
//   s_jm = tanh'(.) z_jm + tanh''(.) z_j z_m,
// with tanh' = 1 - a^2, tanh'' = -2 a (1 - a^2).  The input layer needs no
// GEMM (its tangents are W_0's columns, its second derivatives zero before
// the activation) and the 3-row output layer is a reduction per column.
#include <algorithm>

#include "rtn_internal.cuh"

namespace rtn {
namespace {

constexpr int C2 = 1 + NZ + NZ * (NZ + 1) / 2;  // 171 columns per node

// column 18 + p of a node holds the pair (j, m), j <= m, in row-major upper
// triangle order
__constant__ unsigned char k_pj[NZ * (NZ + 1) / 2];
__constant__ unsigned char k_pm[NZ * (NZ + 1) / 2];

// input layer: one thread per (neuron i, node n, column c)
__global__ void h2_in_kernel(const float* __restrict__ x, const float* __restrict__ u,
                             const int* __restrict__ node_inst, int n_nodes, const float* __restrict__ W0,
                             const float* __restrict__ b0, int h0, float* __restrict__ X1) {
  const long long cols = (long long)C2 * n_nodes;
  const long long total = (long long)h0 * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / cols);
    const long long rem = e % cols;
    const int n = (int)(rem / C2), c = (int)(rem % C2);
    const float* xr = x + (size_t)(n + node_inst[n]) * NX;
    const float* ur = u + (size_t)n * NU;
    const float* w = W0 + (size_t)i * NZ;
    float s = b0[i];
#pragma unroll
    for (int j = 0; j < NX; ++j) s = fmaf(w[j], xr[j], s);
#pragma unroll
    for (int j = 0; j < NU; ++j) s = fmaf(w[NX + j], ur[j], s);
    const float a = tanhf(s), d1 = 1.0f - a * a, d2 = -2.0f * a * d1;
    float v;
    if (c == 0) v = a;
    else if (c <= NZ) v = d1 * w[c - 1];
    else v = d2 * w[k_pj[c - 1 - NZ]] * w[k_pm[c - 1 - NZ]];
    X1[(size_t)i * cols + rem] = v;
  }
}

// C [M][N] = A [M][K] B [K][N], row-major FP32; 64 x 64 tiles, 16 K per step,
// 256 threads computing 4 x 4 each
__global__ void __launch_bounds__(256) h2_gemm_kernel(const float* __restrict__ A, const float* __restrict__ B,
                                                      float* __restrict__ Cm, int M, int N, int K) {
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;
  for (int k0 = 0; k0 < K; k0 += 16) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = threadIdx.x + 256 * r;
      // A tile: 64 rows x 16 k (k fastest), stored transposed
      const int am = e >> 4, ak = e & 15;
      As[ak][am] = (m0 + am < M && k0 + ak < K) ? __ldg(A + (size_t)(m0 + am) * K + k0 + ak) : 0.0f;
      // B tile: 16 k x 64 columns (columns fastest)
      const int bk = e >> 6, bn = e & 63;
      Bs[bk][bn] = (k0 + bk < K && n0 + bn < N) ? __ldg(B + (size_t)(k0 + bk) * N + n0 + bn) : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[kk][ty * 4 + a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx * 4 + b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int m = m0 + ty * 4 + a;
    if (m >= M) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int n = n0 + tx * 4 + b;
      if (n < N) Cm[(size_t)m * N + n] = acc[a][b];
    }
  }
}

// hidden-layer activation: one thread per (neuron i, node n, column c)
__global__ void h2_act_kernel(const float* __restrict__ Z, const float* __restrict__ bias, int h,
                              int n_nodes, float* __restrict__ X) {
  const long long cols = (long long)C2 * n_nodes;
  const long long total = (long long)h * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / cols);
    const long long rem = e % cols;
    const int c = (int)(rem % C2);
    const float* z = Z + (size_t)i * cols + (rem - c);  // the node's 171 columns
    const float a = tanhf(z[0] + bias[i]), d1 = 1.0f - a * a, d2 = -2.0f * a * d1;
    float v;
    if (c == 0) v = a;
    else if (c <= NZ) v = d1 * z[c];
    else {
      const int p = c - 1 - NZ;
      v = fmaf(d2, z[1 + k_pj[p]] * z[1 + k_pm[p]], d1 * z[c]);
    }
    X[(size_t)i * cols + rem] = v;
  }
}

// output layer (linear, NOUT = 3 or 6 rows): one thread per (node n, column
// c); writes f_D [n][NOUT], J_D [n][NOUT][17] and H_D [n][NOUT][17][17]
// (both triangles)
template <int NOUT>
__global__ void h2_out_kernel(const float* __restrict__ WL, const float* __restrict__ bL, int h, int n_nodes,
                              const float* __restrict__ X, float* __restrict__ fD, float* __restrict__ JD,
                              float* __restrict__ HD) {
  const long long cols = (long long)C2 * n_nodes;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < cols;
       e += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(e / C2), c = (int)(e % C2);
    float acc[NOUT];
#pragma unroll
    for (int r = 0; r < NOUT; ++r) acc[r] = 0.0f;
    for (int k = 0; k < h; ++k) {
      const float xv = __ldg(X + (size_t)k * cols + e);
#pragma unroll
      for (int r = 0; r < NOUT; ++r) acc[r] = fmaf(__ldg(WL + (size_t)r * h + k), xv, acc[r]);
    }
#pragma unroll
    for (int r = 0; r < NOUT; ++r) {
      if (c == 0) {
        fD[(size_t)n * NOUT + r] = acc[r] + bL[r];
      } else if (c <= NZ) {
        JD[((size_t)n * NOUT + r) * NZ + (c - 1)] = acc[r];
      } else {
        const int p = c - 1 - NZ, j = k_pj[p], m = k_pm[p];
        float* Hr = HD + ((size_t)n * NOUT + r) * NZ * NZ;
        Hr[j * NZ + m] = acc[r];
        Hr[m * NZ + j] = acc[r];
      }
    }
  }
}

int grid_for(long long work) {
  return (int)std::min<long long>((work + 255) / 256, 148LL * 32);
}

}  // namespace

// the (j, m) pair table of the second-order columns (at context creation:
// the forward pass itself stays capturable in a CUDA graph)
cudaError_t mlp_hess_prepare() {
  unsigned char pj[NZ * (NZ + 1) / 2], pm[NZ * (NZ + 1) / 2];
  int p = 0;
  for (int j = 0; j < NZ; ++j)
    for (int m = j; m < NZ; ++m) {
      pj[p] = (unsigned char)j;
      pm[p] = (unsigned char)m;
      ++p;
    }
  cudaError_t e = cudaMemcpyToSymbol(k_pj, pj, sizeof(pj));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(k_pm, pm, sizeof(pm));
  return e;
}

size_t mlp_hess_act_floats(const rtn_ctx* ctx) {
  return (size_t)ctx->net.h_max * C2 * ctx->lay.n_nodes;
}

cudaError_t mlp_hess_forward(rtn_ctx* ctx, const float* x, const float* u, float* fD, float* JD, float* HD) {
  Net& net = ctx->net;
  const int n = ctx->lay.n_nodes, L = net.n_layers;
  cudaStream_t s = ctx->stream;
  const long long cols = (long long)C2 * n;
  const int h1 = net.widths[1];
  h2_in_kernel<<<grid_for((long long)h1 * cols), 256, 0, s>>>(x, u, ctx->lay.node_inst, n, net.W32 + net.w_off[0],
                                                             net.b32 + net.b_off[0], h1, ctx->h2_x);
  for (int l = 1; l + 1 < L; ++l) {
    const int hi = net.widths[l], ho = net.widths[l + 1];
    dim3 grid((unsigned)((cols + 63) / 64), (unsigned)((ho + 63) / 64));
    h2_gemm_kernel<<<grid, 256, 0, s>>>(net.W32 + net.w_off[l], ctx->h2_x, ctx->h2_z, ho, (int)cols, hi);
    h2_act_kernel<<<grid_for((long long)ho * cols), 256, 0, s>>>(ctx->h2_z, net.b32 + net.b_off[l], ho, n,
                                                                  ctx->h2_x);
  }
  auto out = net.widths[L] == NO_FULL ? h2_out_kernel<NO_FULL> : h2_out_kernel<NO>;
  out<<<grid_for(cols), 256, 0, s>>>(net.W32 + net.w_off[L - 1], net.b32 + net.b_off[L - 1], net.widths[L - 1], n,
                                     ctx->h2_x, fD, JD, HD);
  return cudaGetLastError();
}

}  // namespace rtn
