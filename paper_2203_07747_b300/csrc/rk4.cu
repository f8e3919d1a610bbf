// rk4.cu -- (a2) the RK4 discretisation of f_F + f_D* with its sensitivities
// A_k, B_k and the defect c_k (Eq. 2) for every node: one thread per (node,
// column of [A | B]); the device code (Eq. 6 dynamics, their directional
// derivatives, the four stages) is in rk4_dev.cuh.
#include "rk4_dev.cuh"

namespace rtn {
namespace {

template <int NOUT>
__global__ void __launch_bounds__(256, 2) rk4_sens_kernel(
    QuadParams P, const float* __restrict__ x, const float* __restrict__ u,
    const float* __restrict__ fD, const float* __restrict__ JD, const float* __restrict__ HD,
    const int* __restrict__ node_inst,
    const float* __restrict__ dt_inst, int n_nodes, float* __restrict__ A, float* __restrict__ Bm,
    float* __restrict__ c) {
  long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (long long)n_nodes * NZ) return;
  rk4_column<NOUT>(P, x, u, fD, JD, HD, node_inst, dt_inst, (int)(tid / NZ), (int)(tid % NZ), A, Bm, c);
}

}  // namespace

cudaError_t rk4_sens(rtn_ctx* ctx, const float* x, const float* u, const float* fD,
                     const float* JD, const float* HD, float* A, float* Bm, float* c) {
  const int nn = ctx->lay.n_nodes;
  long long tot = (long long)nn * NZ;
  auto kern = ctx->n_out == NO_FULL ? rk4_sens_kernel<NO_FULL> : rk4_sens_kernel<NO>;
  kern<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(ctx->quad, x, u, fD, JD, fD ? HD : nullptr,
                                                                ctx->lay.node_inst, ctx->lay.dt, nn, A, Bm, c);
  return cudaGetLastError();
}

}  // namespace rtn
