// rk4_dev.cuh -- (a2) device code of the RK4 discretisation of f_F + f_D*
// with its sensitivities, shared by the RK4 kernel (rk4.cu) and the fused
// linearisation + QP kernel of the ragged batch (riccati.cu).  Internal to
// librtn.
//
// For node k the continuity condition of Eq. 2 needs phi_k = RK4(x_k, u_k),
// A_k = dphi/dx and B_k = dphi/du (Sec. III-A), where the dynamics are the
// nominal quadrotor model of Eq. 6 plus the local model of the residual
// (Eq. 4), f_D*(x, u) = fbar + J_D dz (+ 1/2 dz' H_r dz for the second-order
// model), dz = [x - x_k; u - u_k]; NOUT = 3 outputs are added to dv/dt, 6
// (the full residual of Eq. 7) to dv/dt and dw/dt -- row r to component 7 + r.  u is held over the
// interval, so dz has no input part at the stage points.
//
// One thread per (node, column j of [A | B]): the thread integrates the node
// and carries one sensitivity direction d(stage)/d z_j through the four
// stages as a Jacobian-vector product of the dynamics, so 17 threads produce
// the 17 columns with no inter-thread traffic.  Consecutive threads write
// consecutive columns of a row of A (and B), which keeps the stores coalesced.
#pragma once

#include "rtn_internal.cuh"

namespace rtn {
namespace {

__device__ __forceinline__ void qmul(const float* a, const float* b, float* r) {
  r[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  r[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
  r[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
  r[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

// third column of the (unnormalised) rotation q (.) e_z = q (0,0,0,1) q^*
__device__ __forceinline__ void rot_ez(const float* q, float* r) {
  r[0] = 2.0f * (q[1] * q[3] + q[0] * q[2]);
  r[1] = 2.0f * (q[2] * q[3] - q[0] * q[1]);
  r[2] = q[0] * q[0] - q[1] * q[1] - q[2] * q[2] + q[3] * q[3];
}

// Eq. 6: nominal dynamics
__device__ __forceinline__ void f_nominal(const QuadParams& P, const float* x, const float* u,
                                          float* xd) {
  xd[0] = x[7]; xd[1] = x[8]; xd[2] = x[9];
  float w[4] = {0.0f, 0.5f * x[10], 0.5f * x[11], 0.5f * x[12]};
  qmul(x + 3, w, xd + 3);
  float T = (u[0] + u[1]) + (u[2] + u[3]);
  float r[3];
  rot_ez(x + 3, r);
  xd[7] = T * P.inv_mass * r[0];
  xd[8] = T * P.inv_mass * r[1];
  xd[9] = T * P.inv_mass * r[2] - P.g;
  // J^-1 (tau - w x J w) with J^-1 folded into the coefficients
  const float wx = x[10], wy = x[11], wz = x[12];
  xd[10] = P.tq[0] * ((u[2] + u[3]) - (u[0] + u[1])) - P.gy[0] * wy * wz;
  xd[11] = P.tq[1] * ((u[1] + u[2]) - (u[0] + u[3])) - P.gy[1] * wz * wx;
  xd[12] = P.tq[2] * ((u[1] + u[3]) - (u[0] + u[2])) - P.gy[2] * wx * wy;
}

// directional derivative of f_nominal at (x, u) along (dx, du)
__device__ __forceinline__ void jvp_nominal(const QuadParams& P, const float* x, const float* u,
                                            const float* dx, const float* du, float* o) {
  o[0] = dx[7]; o[1] = dx[8]; o[2] = dx[9];
  // d(1/2 q (x) (0,w)) = 1/2 (dq (x) (0,w) + q (x) (0,dw))
  float w[4] = {0.0f, 0.5f * x[10], 0.5f * x[11], 0.5f * x[12]};
  float dw[4] = {0.0f, 0.5f * dx[10], 0.5f * dx[11], 0.5f * dx[12]};
  float t1[4], t2[4];
  qmul(dx + 3, w, t1);
  qmul(x + 3, dw, t2);
#pragma unroll
  for (int i = 0; i < 4; ++i) o[3 + i] = t1[i] + t2[i];
  // d((T/m) r(q)) = (dT/m) r + (T/m) dr
  const float* q = x + 3;
  const float* dq = dx + 3;
  float T = (u[0] + u[1]) + (u[2] + u[3]);
  float dT = (du[0] + du[1]) + (du[2] + du[3]);
  float r[3], dr[3];
  rot_ez(q, r);
  dr[0] = 2.0f * (dq[1] * q[3] + q[1] * dq[3] + dq[0] * q[2] + q[0] * dq[2]);
  dr[1] = 2.0f * (dq[2] * q[3] + q[2] * dq[3] - dq[0] * q[1] - q[0] * dq[1]);
  dr[2] = 2.0f * (q[0] * dq[0] - q[1] * dq[1] - q[2] * dq[2] + q[3] * dq[3]);
#pragma unroll
  for (int i = 0; i < 3; ++i) o[7 + i] = P.inv_mass * (dT * r[i] + T * dr[i]);
  // d(J^-1 (tau - w x J w))
  const float wx = x[10], wy = x[11], wz = x[12], dwx = dx[10], dwy = dx[11], dwz = dx[12];
  o[10] = P.tq[0] * ((du[2] + du[3]) - (du[0] + du[1])) - P.gy[0] * (dwy * wz + wy * dwz);
  o[11] = P.tq[1] * ((du[1] + du[2]) - (du[0] + du[3])) - P.gy[1] * (dwz * wx + wz * dwx);
  o[12] = P.tq[2] * ((du[1] + du[3]) - (du[0] + du[2])) - P.gy[2] * (dwx * wy + wx * dwy);
}

// node n, column j of [A | B] (j = 0 also writes c_n)
template <int NOUT>
__device__ __forceinline__ void rk4_column(
    const QuadParams& P, const float* __restrict__ x, const float* __restrict__ u,
    const float* __restrict__ fD, const float* __restrict__ JD, const float* __restrict__ HD,
    const int* __restrict__ node_inst, const float* __restrict__ dt_inst, int n, int j,
    float* __restrict__ A, float* __restrict__ Bm, float* __restrict__ c) {
  const int b = node_inst[n];
  const float h = dt_inst[b];
  const float* xk = x + (size_t)(n + b) * NX;
  float x0[NX], uk[NU], fb[NOUT];
  // J_D is read from L1 where it is used (the 17 threads of a node share it)
  // rather than held in registers: half the registers, twice the resident warps
  const float* __restrict__ Jp = JD ? JD + (size_t)n * NOUT * NZ : nullptr;
#pragma unroll
  for (int i = 0; i < NX; ++i) x0[i] = xk[i];
#pragma unroll
  for (int i = 0; i < NU; ++i) uk[i] = u[(size_t)n * NU + i];
  bool res = fD != nullptr;
  if (res) {
    bool fin = true;
#pragma unroll
    for (int r = 0; r < NOUT; ++r) {
      fb[r] = fD[(size_t)n * NOUT + r];
      fin &= isfinite(fb[r]);
      for (int i = 0; i < NZ; ++i) fin &= isfinite(__ldg(Jp + r * NZ + i));
    }
    res = fin;  // non-finite residual: fall back to the nominal model
  }
  // direction of this thread: e_j in [x; u]
  float du[NU], S[NX];
#pragma unroll
  for (int i = 0; i < NU; ++i) du[i] = (j == NX + i) ? 1.0f : 0.0f;
#pragma unroll
  for (int i = 0; i < NX; ++i) S[i] = (i == j) ? 1.0f : 0.0f;
  // at the first stage (xs = x0, Ss = e_j) the local model's value is f_D
  // itself and its directional derivative the entry J_D[r][j]: exact, the
  // results of the full products bit for bit, without their 17 loads
  float xs[NX], Ss[NX], k[NX], dk[NX], ksum[NX], dksum[NX];
#pragma unroll
  for (int i = 0; i < NX; ++i) { ksum[i] = 0.0f; dksum[i] = 0.0f; }
  const float cst[4] = {0.0f, 0.5f, 0.5f, 1.0f};
  const float wgt[4] = {1.0f, 2.0f, 2.0f, 1.0f};
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    if (s == 0) {
#pragma unroll
      for (int i = 0; i < NX; ++i) { xs[i] = x0[i]; Ss[i] = S[i]; }
    } else {
#pragma unroll
      for (int i = 0; i < NX; ++i) {
        xs[i] = fmaf(cst[s] * h, k[i], x0[i]);
        Ss[i] = fmaf(cst[s] * h, dk[i], S[i]);
      }
    }
    f_nominal(P, xs, uk, k);
    jvp_nominal(P, xs, uk, Ss, du, dk);
    if (res) {
#pragma unroll
      for (int r = 0; r < NOUT; ++r) {
        float v = fb[r], dv;
        if (s == 0) {
          dv = __ldg(Jp + r * NZ + j);
        } else {
          dv = 0.0f;
#pragma unroll
          for (int i = 0; i < NX; ++i) {
            const float Jri = __ldg(Jp + r * NZ + i);
            v = fmaf(Jri, xs[i] - x0[i], v);
            dv = fmaf(Jri, Ss[i], dv);
          }
#pragma unroll
          for (int i = 0; i < NU; ++i) dv = fmaf(__ldg(Jp + r * NZ + NX + i), du[i], dv);
        }
        if (HD && s > 0) {
          // g = H_r dz (dz = xs - x0 on the state part): value + 1/2 dz'g,
          // directional derivative + g . [S; du]
          const float* Hr = HD + ((size_t)n * NOUT + r) * NZ * NZ;
          float q = 0.0f;
          for (int i = 0; i < NZ; ++i) {
            float g = 0.0f;
#pragma unroll
            for (int m = 0; m < NX; ++m) g = fmaf(__ldg(Hr + i * NZ + m), xs[m] - x0[m], g);
            if (i < NX) {
              q = fmaf(0.5f * (xs[i] - x0[i]), g, q);
              dv = fmaf(g, Ss[i], dv);
            } else {
              dv = fmaf(g, du[i - NX], dv);
            }
          }
          v += q;
        }
        k[7 + r] += v;
        dk[7 + r] += dv;
      }
    }
#pragma unroll
    for (int i = 0; i < NX; ++i) {
      ksum[i] = fmaf(wgt[s], k[i], ksum[i]);
      dksum[i] = fmaf(wgt[s], dk[i], dksum[i]);
    }
  }
  const float h6 = h / 6.0f;
  if (j < NX) {
    float* a = A + (size_t)n * NX * NX + j;
#pragma unroll
    for (int i = 0; i < NX; ++i) a[i * NX] = S[i] + h6 * dksum[i];
  } else {
    float* bb = Bm + (size_t)n * NX * NU + (j - NX);
#pragma unroll
    for (int i = 0; i < NX; ++i) bb[i * NU] = h6 * dksum[i];
  }
  if (j == 0) {
    const float* xn = xk + NX;
#pragma unroll
    for (int i = 0; i < NX; ++i) c[(size_t)n * NX + i] = (x0[i] + h6 * ksum[i]) - xn[i];
  }
}


}  // namespace
}  // namespace rtn
