// riccati.cu -- (a3) + (a4): the linear-quadratic subproblem of Sec. III-A and
// the feedback response of Sec. III-B, for every instance of the batch.
//
//   min  sum_k 1/2 dx'Q dx + q_k'dx + 1/2 du'R du + r_k'du + 1/2 dxN'QN dxN + pN'dxN
//   s.t. dx_0 = x0_meas - x_0,   dx_{k+1} = A_k dx_k + B_k du_k + c_k     (Eq. 2)
// with the Gauss-Newton terms of the quadratic tracking cost of Sec. V:
// q_k = Q (x_k - xr_k), r_k = R (u_k - ur_k), pN = QN (x_N - xr_N).
//
// Backward Riccati sweep (sequential over k, parallel over instances):
//   Huu = R + B'PB, Hux = B'PA, hu = r + B'(p + Pc)
//   [K | k] = -Huu^{-1} [Hux | hu]            (Cholesky of Huu in FP64)
//   P <- Q + A'PA + Hux'K (symmetrised),  p <- q + A'(p + Pc) + Hux'k
// Forward: du_k = K dx_k + k,  dx_{k+1} = A dx_k + B du_k + c.
// The feedback response then updates the iterate (w += dw), sends
// u_0 = clamp(u_0 + du_0, 0, u_max) and shifts the iterate by one stage.
//
// One warp per instance; the 13x13 / 13x4 / 4x4 blocks live in the warp's
// shared-memory slot and the lanes share each matrix product element-wise.
// Instances are visited longest-horizon first so that the ragged tail of a
// batch with uneven N_b finishes together.
#include "rtn_internal.cuh"

namespace rtn {
namespace {

template <typename T>
struct Slot {
  T A[NX * NX], Bm[NX * NU], c[NX];
  T P[NX * NX], p[NX];
  T PA[NX * NX], PB[NX * NU], g[NX];
  T Huu[NU * NU], Hux[NU * NX], hu[NU];
  T K[NU * NX], k[NU];
  T P2[NX * NX], p2[NX];
  T dx[NX], du[NU];
  double L[NU * NU], Linv[NU];  // FP64 Cholesky factor (strict lower part) and 1/diag
  int notpd;
};

struct KArgs {
  QpArgs a;
  CostParams cost;
  float u_max;
  int B;
  const int *N, *xoff, *uoff, *order;
  void* Kg;  // [n_nodes][4][13] of T
  void* kg;  // [n_nodes][4] of T
};

template <typename T, int WPB>
__global__ void __launch_bounds__(WPB * 32) qp_kernel(KArgs ka) {
  __shared__ Slot<T> slots[WPB];
  const QpArgs& a = ka.a;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int slot = blockIdx.x * WPB + warp;
  if (slot >= ka.B) return;
  const int b = ka.order ? ka.order[slot] : slot;
  Slot<T>& S = slots[warp];
  const int N = ka.N[b], xo = ka.xoff[b], uo = ka.uoff[b];
  const int t = a.t_dev ? *a.t_dev : 0;
  const int xr0 = (a.xref_stride > 0 ? b * a.xref_stride : xo) + t;
  const int ur0 = (a.uref_stride > 0 ? b * a.uref_stride : uo) + t;
  const float* x = a.x + (size_t)xo * NX;
  const float* u = a.u + (size_t)uo * NU;
  const float* xr = a.xref + (size_t)xr0 * NX;
  const float* ur = a.uref + (size_t)ur0 * NU;
  T* Kg = reinterpret_cast<T*>(ka.Kg);
  T* kg = reinterpret_cast<T*>(ka.kg);
  const CostParams& C = ka.cost;

  // measured state
  float x0m = lane < NX ? a.x0[(size_t)b * NX + lane] : 0.0f;
  const bool finite = __all_sync(0xffffffffu, isfinite(x0m));

  for (int e = lane; e < NX * NX; e += 32) {
    int i = e / NX, j = e % NX;
    S.P[e] = (i == j) ? (T)C.QN[i] : (T)0;
  }
  if (lane < NX)
    S.p[lane] = (T)C.QN[lane] * ((T)x[(size_t)N * NX + lane] - (T)xr[(size_t)N * NX + lane]);
  if (lane == 0) S.notpd = 0;
  __syncwarp();

  for (int k = N - 1; k >= 0 && finite; --k) {
    const size_t node = (size_t)uo + k;
    const float* Ak = a.A + node * NX * NX;
    const float* Bk = a.Bm + node * NX * NU;
    const float* ck = a.c + node * NX;
    for (int e = lane; e < NX * NX; e += 32) S.A[e] = (T)Ak[e];
    for (int e = lane; e < NX * NU; e += 32) S.Bm[e] = (T)Bk[e];
    if (lane < NX) S.c[lane] = (T)ck[lane];
    __syncwarp();
    // PA = P A, PB = P B, g = p + P c
    for (int e = lane; e < NX * NX + NX * NU + NX; e += 32) {
      if (e < NX * NX) {
        int i = e / NX, j = e % NX;
        T s = 0;
#pragma unroll
        for (int l = 0; l < NX; ++l) s += S.P[i * NX + l] * S.A[l * NX + j];
        S.PA[e] = s;
      } else if (e < NX * NX + NX * NU) {
        int f = e - NX * NX, i = f / NU, j = f % NU;
        T s = 0;
#pragma unroll
        for (int l = 0; l < NX; ++l) s += S.P[i * NX + l] * S.Bm[l * NU + j];
        S.PB[f] = s;
      } else {
        int i = e - NX * NX - NX * NU;
        T s = S.p[i];
#pragma unroll
        for (int l = 0; l < NX; ++l) s += S.P[i * NX + l] * S.c[l];
        S.g[i] = s;
      }
    }
    __syncwarp();
    // Huu = R + B'PB, Hux = B'PA, hu = r + B'g
    for (int e = lane; e < NU * NU + NU * NX + NU; e += 32) {
      if (e < NU * NU) {
        int i = e / NU, j = e % NU;
        T s = (i == j) ? (T)C.R[i] : (T)0;
#pragma unroll
        for (int l = 0; l < NX; ++l) s += S.Bm[l * NU + i] * S.PB[l * NU + j];
        S.Huu[e] = s;
      } else if (e < NU * NU + NU * NX) {
        int f = e - NU * NU, i = f / NX, j = f % NX;
        T s = 0;
#pragma unroll
        for (int l = 0; l < NX; ++l) s += S.Bm[l * NU + i] * S.PA[l * NX + j];
        S.Hux[f] = s;
      } else {
        int i = e - NU * NU - NU * NX;
        T s = (T)C.R[i] * ((T)u[(size_t)k * NU + i] - (T)ur[(size_t)k * NU + i]);
#pragma unroll
        for (int l = 0; l < NX; ++l) s += S.Bm[l * NU + i] * S.g[l];
        S.hu[i] = s;
      }
    }
    __syncwarp();
    // FP64 Cholesky of Huu by one lane (4 square roots, 4 reciprocals), then
    // the 14 right-hand sides (13 of Hux, 1 of hu) on 14 lanes with products
    if (lane == 0) {
      double L[NU][NU];
      bool pd = true;
#pragma unroll
      for (int j = 0; j < NU; ++j) {
        double s = (double)S.Huu[j * NU + j];
#pragma unroll
        for (int q = 0; q < j; ++q) s -= L[j][q] * L[j][q];
        pd &= (s > 0.0);
        const double d = sqrt(fmax(s, 1e-300)), inv = 1.0 / d;
        L[j][j] = d;
        S.Linv[j] = inv;
#pragma unroll
        for (int i = j + 1; i < NU; ++i) {
          double v = (double)S.Huu[i * NU + j];
#pragma unroll
          for (int q = 0; q < j; ++q) v -= L[i][q] * L[j][q];
          L[i][j] = v * inv;
        }
      }
#pragma unroll
      for (int i = 0; i < NU; ++i)
#pragma unroll
        for (int j = 0; j < NU; ++j) S.L[i * NU + j] = (j < i) ? L[i][j] : 0.0;
      if (!pd) S.notpd = 1;
    }
    __syncwarp();
    if (lane < NX + 1) {
      double y[NU];
#pragma unroll
      for (int i = 0; i < NU; ++i) {
        double v = (lane < NX) ? (double)S.Hux[i * NX + lane] : (double)S.hu[i];
#pragma unroll
        for (int q = 0; q < i; ++q) v -= S.L[i * NU + q] * y[q];
        y[i] = v * S.Linv[i];
      }
#pragma unroll
      for (int i = NU - 1; i >= 0; --i) {
        double v = y[i];
#pragma unroll
        for (int q = i + 1; q < NU; ++q) v -= S.L[q * NU + i] * y[q];
        y[i] = v * S.Linv[i];
      }
#pragma unroll
      for (int i = 0; i < NU; ++i) {
        if (lane < NX) S.K[i * NX + lane] = (T)(-y[i]);
        else S.k[i] = (T)(-y[i]);
      }
    }
    __syncwarp();
    // P2 = Q + A'PA + Hux'K,  p2 = q + A'g + Hux'k ; store the gains
    for (int e = lane; e < NX * NX + NX; e += 32) {
      if (e < NX * NX) {
        int i = e / NX, j = e % NX;
        T s = (i == j) ? (T)C.Q[i] : (T)0;
#pragma unroll
        for (int l = 0; l < NX; ++l) s += S.A[l * NX + i] * S.PA[l * NX + j];
#pragma unroll
        for (int l = 0; l < NU; ++l) s += S.Hux[l * NX + i] * S.K[l * NX + j];
        S.P2[e] = s;
      } else {
        int i = e - NX * NX;
        T s = (T)C.Q[i] * ((T)x[(size_t)k * NX + i] - (T)xr[(size_t)k * NX + i]);
#pragma unroll
        for (int l = 0; l < NX; ++l) s += S.A[l * NX + i] * S.g[l];
#pragma unroll
        for (int l = 0; l < NU; ++l) s += S.Hux[l * NX + i] * S.k[l];
        S.p2[i] = s;
      }
    }
    for (int e = lane; e < NU * NX + NU; e += 32) {
      if (e < NU * NX) Kg[node * NU * NX + e] = S.K[e];
      else kg[node * NU + (e - NU * NX)] = S.k[e - NU * NX];
    }
    __syncwarp();
    for (int e = lane; e < NX * NX + NX; e += 32) {
      if (e < NX * NX) {
        int i = e / NX, j = e % NX;
        S.P[e] = (T)0.5 * (S.P2[i * NX + j] + S.P2[j * NX + i]);
      } else {
        S.p[e - NX * NX] = S.p2[e - NX * NX];
      }
    }
    __syncwarp();
  }

  const int st = !finite ? RTN_E_NONFINITE : (S.notpd ? RTN_E_NOT_PD : RTN_OK);
  if (lane == 0 && a.status) a.status[b] = st;
  if (st != RTN_OK) {
    // failed instance: zero step, iterate untouched, send the reference input
    if (a.dx)
      for (int e = lane; e < (N + 1) * NX; e += 32) a.dx[(size_t)xo * NX + e] = 0.0f;
    if (a.du)
      for (int e = lane; e < N * NU; e += 32) a.du[(size_t)uo * NU + e] = 0.0f;
    if (a.u0 && lane < NU) a.u0[(size_t)b * NU + lane] = ur[lane];
    return;
  }

  // forward roll-out and feedback response.  Lane i only ever touches
  // component i of a row, so the in-place update needs no cross-lane ordering:
  // row k+1 of the old iterate is read before row k+1 is rewritten.
  float* xw = a.x + (size_t)xo * NX;
  float* uw = a.u + (size_t)uo * NU;
  if (lane < NX) S.dx[lane] = (T)x0m - (T)x[lane];
  __syncwarp();
  if (a.dx && lane < NX) a.dx[(size_t)xo * NX + lane] = (float)S.dx[lane];
  if (a.update && !a.shift && lane < NX) xw[lane] = (float)((T)x[lane] + S.dx[lane]);
  for (int k = 0; k < N; ++k) {
    const size_t node = (size_t)uo + k;
    if (lane < NU) {
      T s = kg[node * NU + lane];
#pragma unroll
      for (int j = 0; j < NX; ++j) s += Kg[node * NU * NX + lane * NX + j] * S.dx[j];
      S.du[lane] = s;
    }
    __syncwarp();
    T dxn = 0;
    if (lane < NX) {
      const float* Ak = a.A + node * NX * NX + lane * NX;
      const float* Bk = a.Bm + node * NX * NU + lane * NU;
      T s = (T)a.c[node * NX + lane];
#pragma unroll
      for (int j = 0; j < NX; ++j) s += (T)Ak[j] * S.dx[j];
#pragma unroll
      for (int j = 0; j < NU; ++j) s += (T)Bk[j] * S.du[j];
      dxn = s;
    }
    if (lane < NU) {
      T unew = (T)u[(size_t)k * NU + lane] + S.du[lane];
      if (a.du) a.du[node * NU + lane] = (float)S.du[lane];
      if (k == 0 && a.u0) {
        float v = (float)unew;
        a.u0[(size_t)b * NU + lane] = fminf(fmaxf(v, 0.0f), ka.u_max);
      }
      if (a.update) {
        if (a.shift) {
          if (k >= 1) uw[(size_t)(k - 1) * NU + lane] = (float)unew;
          if (k == N - 1) uw[(size_t)k * NU + lane] = (float)unew;
        } else {
          uw[(size_t)k * NU + lane] = (float)unew;
        }
      }
    }
    if (lane < NX) {
      if (a.dx) a.dx[(size_t)(xo + k + 1) * NX + lane] = (float)dxn;
      if (a.update) {
        T xnew = (T)x[(size_t)(k + 1) * NX + lane] + dxn;
        if (a.shift) {
          xw[(size_t)k * NX + lane] = (float)xnew;
          if (k == N - 1) xw[(size_t)(k + 1) * NX + lane] = (float)xnew;
        } else {
          xw[(size_t)(k + 1) * NX + lane] = (float)xnew;
        }
      }
    }
    __syncwarp();
    if (lane < NX) S.dx[lane] = dxn;
    __syncwarp();
  }
}

template <typename T, int WPB>
cudaError_t launch(const KArgs& ka, cudaStream_t s) {
  qp_kernel<T, WPB><<<(ka.B + WPB - 1) / WPB, WPB * 32, 0, s>>>(ka);
  return cudaGetLastError();
}

}  // namespace

cudaError_t qp_solve(rtn_ctx* ctx, const QpArgs& a) {
  KArgs ka;
  ka.a = a;
  ka.cost = ctx->cost;
  ka.u_max = ctx->quad.u_max;
  ka.B = ctx->B;
  ka.N = ctx->lay.N;
  ka.xoff = ctx->lay.xoff;
  ka.uoff = ctx->lay.uoff;
  ka.order = ctx->lay.order;
  ka.Kg = ctx->K;
  ka.kg = ctx->kff;
  if (ctx->opt.riccati_f64) return launch<double, 2>(ka, ctx->stream);
  return launch<float, 4>(ka, ctx->stream);
}

}  // namespace rtn
