// di.cu -- (f3) the runtime-analysis model of Sec. IV on the GPU.
//
// Double integrator x = (p, v), u the commanded acceleration, nominal model
// f_F = (v, u) (Eq. 5), plus a residual network z = (p, v, u) -> one output
// added to dv/dt (in the paper's runtime study its weights are set so that it
// outputs zero; any weights work here).  One RTI step (Sec. III-B):
//   * the network's value f_D and Jacobian J_D (1 x 3) at every node, FP32
//     forward mode (value + 3 tangents = 4 columns per node) -- di_in_kernel
//     (first layer), di_hidden_kernel (hidden -> hidden, any width),
//     di_out_kernel (last layer);
//   * one thread per instance (di_step_kernel, FP32): RK4 of f_F + f_D* with
//     the sensitivities A = dphi/dx, B = dphi/du at every node, the Riccati
//     recursion of the QP (nx = 2, nu = 1), the forward roll-out from the
//     measured x0, the iterate update, u_0, and the shift.
// Layouts follow the quadrotor contexts: states [n_states][2], inputs
// [n_nodes], node-packed ragged instances (Layout).
#include <algorithm>

#include "rtn_internal.cuh"

namespace rtn {
namespace {

constexpr int DI_NC = 4;  // columns per node: value, d/dp, d/dv, d/du

// first layer: a = tanh(W0 z + b0), tangents d * W0[:, j]; one thread per
// (node, unit).  Y: [n_nodes][4][h]
__global__ void di_in_kernel(const float* __restrict__ W0, const float* __restrict__ b0, int h,
                             const float* __restrict__ x, const float* __restrict__ u,
                             const int* __restrict__ node_inst, int n_nodes, float* __restrict__ Y) {
  const long long total = (long long)n_nodes * h;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int node = (int)(idx / h), o = (int)(idx % h);
    const float* xs = x + (size_t)(node + node_inst[node]) * 2;
    const float* w = W0 + (size_t)o * 3;
    float s = b0[o];
    s = fmaf(w[0], xs[0], s);
    s = fmaf(w[1], xs[1], s);
    s = fmaf(w[2], u[node], s);
    const float a = tanhf(s), d = 1.0f - a * a;
    float* y = Y + (size_t)node * DI_NC * h + o;
    y[0] = a;
    y[(size_t)h] = d * w[0];
    y[2 * (size_t)h] = d * w[1];
    y[3 * (size_t)h] = d * w[2];
  }
}

// hidden layer: Y = W X for the 4 columns of 8 nodes and 16 consecutive units
// per 256-thread block (warp w computes units o0 + 2w, o0 + 2w + 1; lanes
// split K), then value a = tanh(y + b), tangents y * (1 - a^2).  The block
// stages its 32 columns of X in shared memory 128 K at a time (independent
// coalesced loads), so every K step of a warp is register/shared-memory
// arithmetic.  X: [n_nodes][4][hi], Y: [n_nodes][4][ho].
constexpr int DI_KC = 128;  // K per staged chunk
constexpr int DI_RO = 2;    // output units per warp

__device__ __forceinline__ void reduce_scatter32(float (&acc)[32], int lane) {
  // butterfly reduce-scatter: lane l ends with the sum of column l in acc[0]
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool up = (lane & s) != 0;
#pragma unroll
    for (int i = 0; i < s; ++i) {
      const float send = up ? acc[i] : acc[i + s];
      const float keep = up ? acc[i + s] : acc[i];
      acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
}

__global__ void __launch_bounds__(256) di_hidden_kernel(const float* __restrict__ W,
                                                        const float* __restrict__ bias, int hi, int ho,
                                                        const float* __restrict__ X,
                                                        float* __restrict__ Y, int n_nodes) {
  __shared__ float xs[32][DI_KC];
  __shared__ float out_s[32][8 * DI_RO + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int o0 = blockIdx.x * 8 * DI_RO;
  const int n0 = blockIdx.y * 8;
  const int ncol = min(8, n_nodes - n0) * DI_NC;  // columns of real nodes
  const float* xb = X + (size_t)n0 * DI_NC * hi;
  float acc[DI_RO][32];
#pragma unroll
  for (int r = 0; r < DI_RO; ++r)
#pragma unroll
    for (int c = 0; c < 32; ++c) acc[r][c] = 0.0f;
  for (int k0 = 0; k0 < hi; k0 += DI_KC) {
    const int kc = min(DI_KC, hi - k0);
    __syncthreads();  // the previous chunk has been used
#pragma unroll
    for (int i = 0; i < 32 * DI_KC / 256; ++i) {
      const int e = threadIdx.x + 256 * i, c = e / DI_KC, kk = e % DI_KC;
      xs[c][kk] = (c < ncol && kk < kc) ? __ldg(xb + (size_t)c * hi + k0 + kk) : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < DI_RO; ++r) {
      const int o = o0 + DI_RO * warp + r;
      if (o >= ho) continue;
      float w[DI_KC / 32];
#pragma unroll
      for (int j = 0; j < DI_KC / 32; ++j)
        w[j] = lane + 32 * j < kc ? __ldg(W + (size_t)o * hi + k0 + lane + 32 * j) : 0.0f;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        float sacc = acc[r][c];
#pragma unroll
        for (int j = 0; j < DI_KC / 32; ++j) sacc = fmaf(w[j], xs[c][lane + 32 * j], sacc);
        acc[r][c] = sacc;
      }
    }
  }
  // column lane = 4 (node - n0) + component
  const int comp = lane & 3;
#pragma unroll
  for (int r = 0; r < DI_RO; ++r) {
    const int o = o0 + DI_RO * warp + r;
    reduce_scatter32(acc[r], lane);
    float a = 0.0f, d = 0.0f;
    if (comp == 0) {
      a = tanhf(acc[r][0] + (o < ho ? bias[o] : 0.0f));
      d = 1.0f - a * a;
    }
    d = __shfl_sync(0xffffffffu, d, lane & ~3);
    out_s[lane][DI_RO * warp + r] = comp == 0 ? a : acc[r][0] * d;
  }
  __syncthreads();
  // 16 consecutive units of each column: one 64-byte run per column
  for (int e = threadIdx.x; e < 32 * 8 * DI_RO; e += 256) {
    const int col = e / (8 * DI_RO), oo = e % (8 * DI_RO);
    if (col < ncol && o0 + oo < ho) Y[((size_t)n0 * DI_NC + col) * ho + o0 + oo] = out_s[col][oo];
  }
}

// last layer (one output, linear): f = W_L a + b_L, J_j = W_L t_j; 4 warps
// per node, warp c the dot product of column c (loads unrolled 4 deep)
__global__ void di_out_kernel(const float* __restrict__ WL, const float* __restrict__ bL, int h,
                              const float* __restrict__ X, int n_nodes, float* __restrict__ fD,
                              float* __restrict__ JD) {
  const int lane = threadIdx.x & 31, c = (threadIdx.x >> 5) & 3;
  const int node = blockIdx.x * (blockDim.x >> 7) + (threadIdx.x >> 7);
  if (node >= n_nodes) return;
  const float* xc = X + ((size_t)node * DI_NC + c) * h;
  float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  int k = lane;
  for (; k + 96 < h; k += 128) {
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] = fmaf(__ldg(WL + k + 32 * j), __ldg(xc + k + 32 * j), acc[j]);
  }
  for (; k < h; k += 32) acc[0] = fmaf(__ldg(WL + k), __ldg(xc + k), acc[0]);
  float s = (acc[0] + acc[1]) + (acc[2] + acc[3]);
#pragma unroll
  for (int sh = 16; sh >= 1; sh >>= 1) s += __shfl_xor_sync(0xffffffffu, s, sh);
  if (lane == 0) {
    if (c == 0) fD[node] = s + bL[0];
    else JD[(size_t)node * 3 + c - 1] = s;
  }
}

int grid_for(long long work, int block) {
  return (int)std::min<long long>((work + block - 1) / block, 148LL * 16);
}

}  // namespace

cudaError_t di_mlp(rtn_ctx* ctx, const float* x, const float* u, float* fD, float* JD) {
  DiState& D = *ctx->di;
  const int n = ctx->lay.n_nodes, L = D.n_layers;
  cudaStream_t s = ctx->stream;
  const int h1 = D.widths[1];
  di_in_kernel<<<grid_for((long long)n * h1, 256), 256, 0, s>>>(D.W + D.w_off[0], D.b + D.b_off[0], h1, x, u,
                                                                 ctx->lay.node_inst, n, D.act0);
  float* cur = D.act0;
  float* nxt = D.act1;
  for (int l = 1; l + 1 < L; ++l) {
    const int hi = D.widths[l], ho = D.widths[l + 1];
    dim3 grid((ho + 8 * DI_RO - 1) / (8 * DI_RO), (n + 7) / 8);
    di_hidden_kernel<<<grid, 256, 0, s>>>(D.W + D.w_off[l], D.b + D.b_off[l], hi, ho, cur, nxt, n);
    std::swap(cur, nxt);
  }
  di_out_kernel<<<(n + 1) / 2, 256, 0, s>>>(D.W + D.w_off[L - 1], D.b + D.b_off[L - 1], D.widths[L - 1],
                                            cur, n, fD, JD);
  return cudaGetLastError();
}

namespace {

// RK4 (u held) of f_F + f_D* with f_D* = fb + J (z - z_k) around the node,
// and the sensitivity S = d(stage)/d[x; u] (2 x 3) through the stages:
// phi = x + dt/6 (k1 + 2 k2 + 2 k3 + k4), A = dphi/dx, B = dphi/du.
template <typename T>
__device__ void di_rk4(const T* x, T u, T fb, const T* J, T dt, T* phi, T* A, T* B) {
  // D = d f / d[p, v, u] (constant: f_F is linear, f_D* affine)
  const T D[6] = {T(0), T(1), T(0), J[0], J[1], T(1) + J[2]};
  const T cst[4] = {T(0), T(0.5), T(0.5), T(1)};
  const T wt[4] = {T(1), T(2), T(2), T(1)};
  T k[2] = {T(0), T(0)}, dk[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
  T ksum[2] = {T(0), T(0)}, dksum[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    T xs[2], S[6];
    for (int i = 0; i < 2; ++i) xs[i] = x[i] + cst[s] * dt * k[i];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 3; ++j) S[i * 3 + j] = ((i == j) ? T(1) : T(0)) + cst[s] * dt * dk[i * 3 + j];
    k[0] = xs[1];
    k[1] = u + fb + J[0] * (xs[0] - x[0]) + J[1] * (xs[1] - x[1]);
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 3; ++j)
        dk[i * 3 + j] = ((j == 2) ? D[i * 3 + 2] : T(0)) + D[i * 3] * S[j] + D[i * 3 + 1] * S[3 + j];
    for (int i = 0; i < 2; ++i) ksum[i] += wt[s] * k[i];
    for (int i = 0; i < 6; ++i) dksum[i] += wt[s] * dk[i];
  }
  const T h6 = dt / T(6);
  for (int i = 0; i < 2; ++i) {
    phi[i] = x[i] + h6 * ksum[i];
    A[i * 2] = (i == 0 ? T(1) : T(0)) + h6 * dksum[i * 3];
    A[i * 2 + 1] = (i == 1 ? T(1) : T(0)) + h6 * dksum[i * 3 + 1];
    B[i] = h6 * dksum[i * 3 + 2];
  }
}

struct DiLay {
  const int* N;
  const float* dt;
  const int* xoff;
  const int* uoff;
  const int* node_inst;
  int B, n_nodes;
};

// linearisation of every node (rtn_linearize): one thread per node
__global__ void di_lin_kernel(DiLay L, const float* __restrict__ x, const float* __restrict__ u,
                              const float* __restrict__ fD, const float* __restrict__ JD, float* A,
                              float* Bm, float* c) {
  const int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= L.n_nodes) return;
  const int b = L.node_inst[node], sx = node + b;  // state row of the node
  const double xk[2] = {x[(size_t)sx * 2], x[(size_t)sx * 2 + 1]};
  double J[3] = {0.0, 0.0, 0.0}, fb = 0.0;
  if (fD) {
    fb = fD[node];
    for (int j = 0; j < 3; ++j) J[j] = JD[(size_t)node * 3 + j];
  }
  double phi[2], Ak[4], Bk[2];
  di_rk4<double>(xk, (double)u[node], fb, J, (double)L.dt[b], phi, Ak, Bk);
  for (int i = 0; i < 4; ++i) A[(size_t)node * 4 + i] = (float)Ak[i];
  for (int i = 0; i < 2; ++i) {
    Bm[(size_t)node * 2 + i] = (float)Bk[i];
    c[(size_t)node * 2 + i] = (float)(phi[i] - x[(size_t)(sx + 1) * 2 + i]);
  }
}

struct DiStepArgs {
  DiLay L;
  const float* fD;   // null: nominal model only
  const float* JD;
  float* x;          // iterate, updated in place
  float* u;
  const float* xref;
  const float* uref;
  const float* x0;   // [B][2] measured states
  float Q[2], QN[2], R;
  float* lin;        // [n_nodes][8] workspace: A (4), B (2), c (2)
  float* K;          // [n_nodes][3] workspace: K (2), k (1)
  float* u0;         // [B]
  int* status;       // [B]
  int shift;
};

// one RTI step of instance b (one thread, FP32): linearise each node (RK4 +
// sensitivities) on the way back through the Riccati recursion, roll out
// from the measured x0 with the stored linearisation, update, u_0, shift
__global__ void di_step_kernel(DiStepArgs a) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.L.B) return;
  const int Nb = a.L.N[b], xo = a.L.xoff[b], uo = a.L.uoff[b];
  const float dt = a.L.dt[b];
  const float x0m[2] = {a.x0[(size_t)b * 2], a.x0[(size_t)b * 2 + 1]};
  if (!isfinite(x0m[0]) || !isfinite(x0m[1])) {
    a.status[b] = RTN_E_NONFINITE;
    a.u0[b] = a.uref[uo];
    return;
  }
  float* xb = a.x + (size_t)xo * 2;
  float* ub = a.u + uo;
  // backward recursion:
  //   P <- Q + A'PA + Hux'K,  p <- q + A'(p + Pc) + Hux'k,
  //   K = -Hux / Huu, k = -hu / Huu  (Huu = R + B'PB scalar)
  float P[4] = {a.QN[0], 0.0f, 0.0f, a.QN[1]};
  float p[2] = {a.QN[0] * (xb[(size_t)Nb * 2] - a.xref[(size_t)(xo + Nb) * 2]),
                a.QN[1] * (xb[(size_t)Nb * 2 + 1] - a.xref[(size_t)(xo + Nb) * 2 + 1])};
  for (int k = Nb - 1; k >= 0; --k) {
    const int nd = uo + k;
    const float xk[2] = {xb[(size_t)k * 2], xb[(size_t)k * 2 + 1]};
    float J[3] = {0.0f, 0.0f, 0.0f}, fb = 0.0f;
    if (a.fD) {
      fb = a.fD[nd];
      for (int j = 0; j < 3; ++j) J[j] = a.JD[(size_t)nd * 3 + j];
    }
    float phi[2], A[4], Bv[2];
    di_rk4<float>(xk, ub[k], fb, J, dt, phi, A, Bv);
    const float c[2] = {phi[0] - xb[(size_t)(k + 1) * 2], phi[1] - xb[(size_t)(k + 1) * 2 + 1]};
    float* ln = a.lin + (size_t)nd * 8;
    for (int i = 0; i < 4; ++i) ln[i] = A[i];
    ln[4] = Bv[0]; ln[5] = Bv[1]; ln[6] = c[0]; ln[7] = c[1];
    float PA[4], PB[2], g[2];
    for (int i = 0; i < 2; ++i) {
      PA[i * 2] = P[i * 2] * A[0] + P[i * 2 + 1] * A[2];
      PA[i * 2 + 1] = P[i * 2] * A[1] + P[i * 2 + 1] * A[3];
      PB[i] = P[i * 2] * Bv[0] + P[i * 2 + 1] * Bv[1];
      g[i] = p[i] + P[i * 2] * c[0] + P[i * 2 + 1] * c[1];
    }
    const float Huu = a.R + Bv[0] * PB[0] + Bv[1] * PB[1];
    const float Hux[2] = {Bv[0] * PA[0] + Bv[1] * PA[2], Bv[0] * PA[1] + Bv[1] * PA[3]};
    const float hu = a.R * (ub[k] - a.uref[nd]) + Bv[0] * g[0] + Bv[1] * g[1];
    if (!(Huu > 0.0f)) {
      a.status[b] = RTN_E_NOT_PD;
      a.u0[b] = a.uref[uo];
      return;
    }
    const float inv = 1.0f / Huu;
    const float Kk[2] = {-Hux[0] * inv, -Hux[1] * inv}, kk = -hu * inv;
    a.K[(size_t)nd * 3] = Kk[0];
    a.K[(size_t)nd * 3 + 1] = Kk[1];
    a.K[(size_t)nd * 3 + 2] = kk;
    float P2[4], p2[2];
    for (int i = 0; i < 2; ++i) {
      for (int j = 0; j < 2; ++j)
        P2[i * 2 + j] = (i == j ? a.Q[i] : 0.0f) + A[i] * PA[j] + A[2 + i] * PA[2 + j] + Hux[i] * Kk[j];
      p2[i] = a.Q[i] * (xk[i] - a.xref[(size_t)(xo + k) * 2 + i]) + A[i] * g[0] + A[2 + i] * g[1] + Hux[i] * kk;
    }
    P[0] = P2[0];
    P[1] = P[2] = 0.5f * (P2[1] + P2[2]);
    P[3] = P2[3];
    p[0] = p2[0];
    p[1] = p2[1];
  }
  // forward roll-out with the stored A, B, c, and the update
  float dx[2] = {x0m[0] - xb[0], x0m[1] - xb[1]};
  for (int k = 0; k < Nb; ++k) {
    const int nd = uo + k;
    const float* ln = a.lin + (size_t)nd * 8;
    const float du = a.K[(size_t)nd * 3 + 2] + a.K[(size_t)nd * 3] * dx[0] + a.K[(size_t)nd * 3 + 1] * dx[1];
    xb[(size_t)k * 2] += dx[0];
    xb[(size_t)k * 2 + 1] += dx[1];
    ub[k] += du;
    const float nx0 = ln[0] * dx[0] + ln[1] * dx[1] + ln[4] * du + ln[6];
    const float nx1 = ln[2] * dx[0] + ln[3] * dx[1] + ln[5] * du + ln[7];
    dx[0] = nx0;
    dx[1] = nx1;
  }
  xb[(size_t)Nb * 2] += dx[0];
  xb[(size_t)Nb * 2 + 1] += dx[1];
  a.u0[b] = ub[0];
  a.status[b] = RTN_OK;
  if (a.shift) {
    for (int k = 0; k < Nb; ++k) {
      xb[(size_t)k * 2] = xb[(size_t)(k + 1) * 2];
      xb[(size_t)k * 2 + 1] = xb[(size_t)(k + 1) * 2 + 1];
    }
    for (int k = 0; k + 1 < Nb; ++k) ub[k] = ub[k + 1];
  }
}

__global__ void di_reset_kernel(DiLay L, const float* __restrict__ x0, float* x, float* u) {
  const int b = blockIdx.x;
  if (b >= L.B) return;
  const int Nb = L.N[b], xo = L.xoff[b], uo = L.uoff[b];
  for (int e = threadIdx.x; e < (Nb + 1) * 2; e += blockDim.x) x[(size_t)xo * 2 + e] = x0[(size_t)b * 2 + e % 2];
  for (int e = threadIdx.x; e < Nb; e += blockDim.x) u[uo + e] = 0.0f;
}

DiLay di_lay(rtn_ctx* ctx) {
  const Layout& L = ctx->lay;
  return DiLay{L.N, L.dt, L.xoff, L.uoff, L.node_inst, L.B, L.n_nodes};
}

}  // namespace

cudaError_t di_linearize(rtn_ctx* ctx, const float* x, const float* u, const float* fD, const float* JD,
                         float* A, float* Bm, float* c) {
  const int n = ctx->lay.n_nodes;
  di_lin_kernel<<<(n + 127) / 128, 128, 0, ctx->stream>>>(di_lay(ctx), x, u, fD, JD, A, Bm, c);
  return cudaGetLastError();
}

cudaError_t di_rti(rtn_ctx* ctx, const float* x0, const float* xref, const float* uref, float* u0,
                   int* status) {
  DiState& D = *ctx->di;
  if (D.n_layers > 0) {
    cudaError_t e = di_mlp(ctx, ctx->x, ctx->u, ctx->fD, ctx->JD);
    if (e != cudaSuccess) return e;
  }
  DiStepArgs a{};
  a.L = di_lay(ctx);
  a.fD = D.n_layers > 0 ? ctx->fD : nullptr;
  a.JD = ctx->JD;
  a.x = ctx->x;
  a.u = ctx->u;
  a.xref = xref;
  a.uref = uref;
  a.x0 = x0;
  a.Q[0] = (float)D.Q[0]; a.Q[1] = (float)D.Q[1];
  a.QN[0] = (float)D.QN[0]; a.QN[1] = (float)D.QN[1];
  a.R = (float)D.R;
  a.lin = D.lin;
  a.K = D.K;
  a.u0 = u0;
  a.status = status ? status : ctx->status;
  a.shift = ctx->opt.shift;
  di_step_kernel<<<(ctx->B + 63) / 64, 64, 0, ctx->stream>>>(a);
  return cudaGetLastError();
}

cudaError_t di_reset(rtn_ctx* ctx, const float* x0) {
  di_reset_kernel<<<ctx->B, 64, 0, ctx->stream>>>(di_lay(ctx), x0, ctx->x, ctx->u);
  return cudaGetLastError();
}

}  // namespace rtn
