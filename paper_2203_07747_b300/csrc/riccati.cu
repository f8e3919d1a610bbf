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
//   [K | k] = -Huu^{-1} [Hux | hu]            (Cholesky of Huu)
//   P <- Q + A'PA + Hux'K (symmetrised),  p <- q + A'(p + Pc) + Hux'k
// Forward: du_k = K dx_k + k,  dx_{k+1} = A dx_k + B du_k + c.
// The feedback response then updates the iterate (w += dw), sends
// u_0 = clamp(u_0 + du_0, 0, u_max) and shifts the iterate by one stage.
//
// One warp per instance, instances visited longest-horizon first so that
// the ragged tail of a batch with uneven N_b finishes together.  In the
// backward sweep lane i < 13 keeps row i of P and p_i in registers; the
// stage matrices and the intermediate products live in the warp's
// shared-memory slot with rows padded to 16 elements, so that every row a
// lane needs whole is read with 16-byte broadcast loads.  The Cholesky of
// Huu (4x4) is computed by one lane and the 14 triangular solves of [K | k]
// on 14 lanes.  Three arithmetic choices (rtn_options.riccati_f64):
//   0  everything in FP32 (Huu is formed in FP32, so a wider factor does
//      not change the error's order, and an FP64 factorisation per node
//      costs more than the rest of the FP32 sweep on this part's FP64 pipe);
//   1  everything in FP64;
//   2  the FP32 sweep with the factorisation of Huu = R + B'PB and the
//      solves of [K | k] in FP64 (FP64 kept only where the QP divides).
#include <algorithm>
#include <type_traits>

#include "rk4_dev.cuh"
#include "rtn_internal.cuh"

namespace rtn {
namespace {

// TC: the type of the factorisation of Huu (its factor is kept rounded to T,
// the type of the solves for [K | k] and of the rest of the sweep)
template <typename T, typename TC>
struct __align__(16) Slot {
  T A[NX][16];    // A_k
  T PA[NX][16];   // P A
  T P2[NX][16];   // next P before symmetrisation
  T Hux[NU][16];  // B'PA
  T K[NU][16];    // feedback gains
  T Bm[NX][NU], PB[NX][NU];
  T c[16], g[16];  // c_k, p + P c
  T Huu[NU * NU], hu[NU], k[NU];
  T Lt[NU * NU], Linvt[NU];  // Cholesky factor of Huu (strict lower part) and 1/diag
  T dx[16], du[NU];
  int notpd;
};

// 16 consecutive elements of a padded shared-memory row into registers
template <typename T>
__device__ __forceinline__ void row16(const T* src, T (&v)[16]) {
  if constexpr (sizeof(T) == 4) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 t = s4[q];
      v[4 * q] = t.x;
      v[4 * q + 1] = t.y;
      v[4 * q + 2] = t.z;
      v[4 * q + 3] = t.w;
    }
  } else {
    const double2* s2 = reinterpret_cast<const double2*>(src);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const double2 t = s2[q];
      v[2 * q] = t.x;
      v[2 * q + 1] = t.y;
    }
  }
}

template <typename T>
__device__ __forceinline__ void row4(const T* src, T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 t = *reinterpret_cast<const float4*>(src);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else {
    const double2* s2 = reinterpret_cast<const double2*>(src);
    const double2 a = s2[0], b = s2[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
}

struct KArgs {
  QpArgs a;
  CostParams cost;
  float u_max;
  int B;
  const int *N, *xoff, *uoff, *order;
  void* Kg;  // [n_nodes][4][13] of T
  void* kg;  // [n_nodes][4] of T
  // box-constrained QP (see rtn_ctx)
  int box, box_max_iter;
  float *box_dx, *box_du, *box_gam;
  signed char* box_act;
  int* box_iters;
};

// Each warp's sweep is one dependent chain, so throughput comes from
// resident warps: at least five blocks per SM (registers capped at 96, a
// few bytes spilled), which at 8192 instances leaves three rounds of warps
// instead of four.
template <typename T, bool CH64>
using SlotOf = Slot<T, typename std::conditional<CH64, double, T>::type>;

// the QP, feedback and iterate update of instance b by a group of G lanes
// (G = 32: one warp; G = 16: a half warp, two instances per warp) with mask
// gm in the warp, lane = the lane's index in the group, and the group's
// shared-memory slot S.  Nothing is exchanged between the groups of a warp.
template <typename T, bool BOX, bool CH64, int G>
__device__ __forceinline__ void qp_instance(const KArgs& ka, int b, SlotOf<T, CH64>& S, int lane, unsigned gm) {
  static_assert(G == 16 || G == 32, "a group is a half warp or a warp");
  using TC = typename std::conditional<CH64, double, T>::type;
  const QpArgs& a = ka.a;
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
  const bool finite = __all_sync(gm, isfinite(x0m));

  // ---------------- backward Riccati sweep (box mode: inputs flagged in
  // box_act are held at their bounds); gains to Kg, kg; S.notpd on failure
  T Prow[NX], p_i = 0;
  auto sweep = [&]() {
#pragma unroll
    for (int j = 0; j < NX; ++j) Prow[j] = (lane < NX && j == lane) ? (T)C.QN[lane] : (T)0;
    if (lane < NX) p_i = (T)C.QN[lane] * ((T)x[(size_t)N * NX + lane] - (T)xr[(size_t)N * NX + lane]);
    if (lane == 0) S.notpd = 0;
    __syncwarp(gm);
    // stage data of node k (A 169, B 52, c 13 floats) as 8 registers per lane,
    // loaded one node ahead so that the global-memory latency overlaps the
    // previous node's arithmetic
    constexpr int NSTAGE = NX * NX + NX * NU + NX;
    constexpr int NPF = (NSTAGE + G - 1) / G;
    float pf[NPF];
    auto prefetch = [&](int k) {
      const size_t node = (size_t)uo + k;
  #pragma unroll
      for (int q = 0; q < NPF; ++q) {
        const int e = lane + G * q;
        float v = 0.0f;
        if (e < NX * NX) v = a.A[node * NX * NX + e];
        else if (e < NX * NX + NX * NU) v = a.Bm[node * NX * NU + (e - NX * NX)];
        else if (e < NSTAGE) v = a.c[node * NX + (e - NX * NX - NX * NU)];
        pf[q] = v;
      }
    };
    if (finite && N > 0) prefetch(N - 1);

    for (int k = N - 1; k >= 0 && finite; --k) {
      const size_t node = (size_t)uo + k;
  #pragma unroll
      for (int q = 0; q < NPF; ++q) {
        const int e = lane + G * q;
        if (e < NX * NX) S.A[e / NX][e % NX] = (T)pf[q];
        else if (e < NX * NX + NX * NU) S.Bm[(e - NX * NX) / NU][(e - NX * NX) % NU] = (T)pf[q];
        else if (e < NSTAGE) S.c[e - NX * NX - NX * NU] = (T)pf[q];
      }
      __syncwarp(gm);
      if (k > 0) prefetch(k - 1);
      // box mode: inputs held at a bound in this subproblem (fx) and their values
      int fx[NU];
      T av[NU];
      {
        const uint32_t w4 = BOX ? *reinterpret_cast<const uint32_t*>(ka.box_act + node * NU) : 0u;
  #pragma unroll
        for (int m = 0; m < NU; ++m) {
          const int v = (int)(signed char)((w4 >> (8 * m)) & 0xffu);
          const T um = (T)u[(size_t)k * NU + m];
          fx[m] = v != 0;
          av[m] = v < 0 ? -um : (v > 0 ? (T)ka.u_max - um : (T)0);
        }
      }
      // PA = P A, PB = P B, g = p + P c: lane i forms row i
      if (lane < NX) {
        T pa[16], pb[NU], gi = p_i;
  #pragma unroll
        for (int j = 0; j < 16; ++j) pa[j] = 0;
  #pragma unroll
        for (int m = 0; m < NU; ++m) pb[m] = 0;
  #pragma unroll
        for (int l = 0; l < NX; ++l) {
          T ar[16], br[4];
          row16(&S.A[l][0], ar);
          row4(&S.Bm[l][0], br);
          const T pl = Prow[l];
  #pragma unroll
          for (int j = 0; j < NX; ++j) pa[j] += pl * ar[j];
  #pragma unroll
          for (int m = 0; m < NU; ++m) pb[m] += pl * br[m];
          gi += pl * S.c[l];
        }
  #pragma unroll
        for (int j = 0; j < NX; ++j) S.PA[lane][j] = pa[j];
  #pragma unroll
        for (int m = 0; m < NU; ++m) S.PB[lane][m] = pb[m];
        S.g[lane] = gi;
      }
      __syncwarp(gm);
      // Hux = B'PA (52), Huu = R + B'PB (16), hu = r + B'g (4) over the warp
      for (int o = lane; o < NU * NX + NU * NU + NU; o += G) {
        T s = 0;
        if (o < NU * NX) {
          const int m = o / NX, j = o % NX;
  #pragma unroll
          for (int l = 0; l < NX; ++l) s += S.Bm[l][m] * S.PA[l][j];
          S.Hux[m][j] = s;
        } else if (o < NU * NX + NU * NU) {
          const int e = o - NU * NX, m = e / NU, n = e % NU;
          s = (m == n) ? (T)C.R[m] : (T)0;
  #pragma unroll
          for (int l = 0; l < NX; ++l) s += S.Bm[l][m] * S.PB[l][n];
          S.Huu[e] = s;
        } else {
          const int m = o - NU * NX - NU * NU;
          s = (T)C.R[m] * ((T)u[(size_t)k * NU + m] - (T)ur[(size_t)k * NU + m]);
  #pragma unroll
          for (int l = 0; l < NX; ++l) s += S.Bm[l][m] * S.g[l];
          S.hu[m] = s;
        }
      }
      __syncwarp(gm);
      if (BOX && lane < NU) ka.box_gam[node * NU + lane] = (float)S.Huu[lane * NU + lane];
      // held inputs: identity rows/columns of Huu, zero rows of Hux, right-hand
      // side -a; their coupling moves to the free rows' right-hand side
      auto Hm = [&](int i, int j) -> TC {
        return (fx[i] || fx[j]) ? (i == j ? (TC)1 : (TC)0) : (TC)S.Huu[i * NU + j];
      };
      // Cholesky of Huu by one lane (one reciprocal square root per pivot)
      if (lane == 0) {
        TC L[NU][NU];
        bool pd = true;
  #pragma unroll
        for (int j = 0; j < NU; ++j) {
          TC s = Hm(j, j);
  #pragma unroll
          for (int q = 0; q < j; ++q) s -= L[j][q] * L[j][q];
          pd &= (s > (TC)0);
          TC inv;
          if constexpr (sizeof(TC) == 4) inv = rsqrtf(fmaxf(s, 1e-30f));
          else inv = rsqrt(fmax(s, 1e-300));
          L[j][j] = s * inv;
          S.Linvt[j] = (T)inv;
  #pragma unroll
          for (int i = j + 1; i < NU; ++i) {
            TC v = Hm(i, j);
  #pragma unroll
            for (int q = 0; q < j; ++q) v -= L[i][q] * L[j][q];
            L[i][j] = v * inv;
          }
        }
  #pragma unroll
        for (int i = 0; i < NU; ++i)
  #pragma unroll
          for (int j = 0; j < NU; ++j) S.Lt[i * NU + j] = (j < i) ? (T)L[i][j] : (T)0;
        if (!pd) S.notpd = 1;
      }
      __syncwarp(gm);
      // [K | k] = -Huu^{-1} [Hux | hu]: right-hand side `lane` (13 = hu)
      if (lane < NX + 1) {
        T y[NU];
  #pragma unroll
        for (int i = 0; i < NU; ++i) {
          T v;
          if (fx[i]) {
            v = (lane < NX) ? (T)0 : -av[i];
          } else {
            v = (lane < NX) ? S.Hux[i][lane] : S.hu[i];
            if (lane == NX) {
  #pragma unroll
              for (int n = 0; n < NU; ++n)
                if (fx[n]) v += S.Huu[i * NU + n] * av[n];
            }
          }
  #pragma unroll
          for (int q = 0; q < i; ++q) v -= S.Lt[i * NU + q] * y[q];
          y[i] = v * S.Linvt[i];
        }
  #pragma unroll
        for (int i = NU - 1; i >= 0; --i) {
          T v = y[i];
  #pragma unroll
          for (int q = i + 1; q < NU; ++q) v -= S.Lt[q * NU + i] * y[q];
          y[i] = v * S.Linvt[i];
        }
  #pragma unroll
        for (int i = 0; i < NU; ++i) {
          if (lane < NX) S.K[i][lane] = -y[i];
          else S.k[i] = -y[i];
        }
      }
      __syncwarp(gm);
      for (int e = lane; e < NU * NX + NU; e += G) {
        if (e < NU * NX) Kg[node * NU * NX + e] = S.K[e / NX][e % NX];
        else kg[node * NU + (e - NU * NX)] = S.k[e - NU * NX];
      }
      // P2 = Q + A'PA + Hux'K (row i on lane i), p2 = q + A'g + Hux'k
      T P2row[16], p2 = 0;
      if (lane < NX) {
  #pragma unroll
        for (int j = 0; j < 16; ++j) P2row[j] = (j == lane) ? (T)C.Q[lane] : (T)0;
        p2 = (T)C.Q[lane] * ((T)x[(size_t)k * NX + lane] - (T)xr[(size_t)k * NX + lane]);
  #pragma unroll
        for (int l = 0; l < NX; ++l) {
          T pr[16];
          row16(&S.PA[l][0], pr);
          const T al = S.A[l][lane];
  #pragma unroll
          for (int j = 0; j < NX; ++j) P2row[j] += al * pr[j];
          p2 += al * S.g[l];
        }
  #pragma unroll
        for (int m = 0; m < NU; ++m) {
          T kr[16];
          row16(&S.K[m][0], kr);
          const T hm = S.Hux[m][lane];
  #pragma unroll
          for (int j = 0; j < NX; ++j) P2row[j] += hm * kr[j];
          p2 += hm * S.k[m];
        }
  #pragma unroll
        for (int j = 0; j < NX; ++j) S.P2[lane][j] = P2row[j];
      }
      __syncwarp(gm);
      if (lane < NX) {
  #pragma unroll
        for (int j = 0; j < NX; ++j) Prow[j] = (T)0.5 * (P2row[j] + S.P2[j][lane]);
        p_i = p2;
      }
      __syncwarp(gm);
    }
  };

  // ---------------- forward roll-out from dx_0 = x0 - x_0.
  //   mode 0: du = K dx + k; step to a.dx/a.du, iterate update, u0 (no bounds)
  //   mode 1: du = K dx + k; step to the box scratch only
  //   mode 2: du from the box scratch (clamped to the bounds if `clamp`);
  //           step to a.dx/a.du, iterate update, u0
  // Lane i only ever touches component i of a row, so the in-place update
  // needs no cross-lane ordering: row k+1 of the old iterate is read before
  // row k+1 is rewritten.
  float* xw = a.x + (size_t)xo * NX;
  float* uw = a.u + (size_t)uo * NU;
  float* bdx = ka.box_dx ? ka.box_dx + (size_t)xo * NX : nullptr;
  float* bdu = ka.box_du ? ka.box_du + (size_t)uo * NU : nullptr;
  auto forward = [&](int mode, bool clamp) {
    const bool final_out = mode != 1;
    if (lane < NX) S.dx[lane] = (T)x0m - (T)x[lane];
    __syncwarp(gm);
    if (lane < NX) {
      if (final_out && a.dx) a.dx[(size_t)xo * NX + lane] = (float)S.dx[lane];
      if (mode == 1) bdx[lane] = (float)S.dx[lane];
      if (final_out && a.update && !a.shift) xw[lane] = (float)((T)x[lane] + S.dx[lane]);
    }
    // per node: lane m < 4 needs its row of K and k (or its stored du); lane
    // i < 13 its rows of A and B and c_i; loaded one node ahead
    float fa[NX], fb[NU], fc = 0.0f;
    T fk[NX], fkk = 0;
    auto fetch = [&](int k) {
      const size_t node = (size_t)uo + k;
      if (lane < NX) {
#pragma unroll
        for (int j = 0; j < NX; ++j) fa[j] = a.A[node * NX * NX + lane * NX + j];
#pragma unroll
        for (int j = 0; j < NU; ++j) fb[j] = a.Bm[node * NX * NU + lane * NU + j];
        fc = a.c[node * NX + lane];
      }
      if (lane < NU) {
        if (mode == 2) {
          fkk = (T)bdu[(size_t)k * NU + lane];
        } else {
#pragma unroll
          for (int j = 0; j < NX; ++j) fk[j] = Kg[node * NU * NX + lane * NX + j];
          fkk = kg[node * NU + lane];
        }
      }
    };
    fetch(0);
    for (int k = 0; k < N; ++k) {
      const size_t node = (size_t)uo + k;
      float ca[NX], cb[NU];
      T ck[NX], ckk = fkk;
      const float cc = fc;
#pragma unroll
      for (int j = 0; j < NX; ++j) { ca[j] = fa[j]; ck[j] = fk[j]; }
#pragma unroll
      for (int j = 0; j < NU; ++j) cb[j] = fb[j];
      if (k + 1 < N) fetch(k + 1);
      if (lane < NU) {
        T s = ckk;
        if (mode == 2) {
          if (clamp) {
            const T um = (T)u[(size_t)k * NU + lane];
            s = fmin(fmax(s, -um), (T)ka.u_max - um);
          }
        } else {
#pragma unroll
          for (int j = 0; j < NX; ++j) s += ck[j] * S.dx[j];
        }
        S.du[lane] = s;
      }
      __syncwarp(gm);
      T dxn = 0;
      if (lane < NX) {
        T s = (T)cc;
#pragma unroll
        for (int j = 0; j < NX; ++j) s += (T)ca[j] * S.dx[j];
#pragma unroll
        for (int j = 0; j < NU; ++j) s += (T)cb[j] * S.du[j];
        dxn = s;
      }
      if (mode == 1) {
        if (lane < NU) bdu[(size_t)k * NU + lane] = (float)S.du[lane];
        if (lane < NX) bdx[(size_t)(k + 1) * NX + lane] = (float)dxn;
      } else {
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
      }
      __syncwarp(gm);
      if (lane < NX) S.dx[lane] = dxn;
      __syncwarp(gm);
    }
  };

  // ---------------- box mode: the cost's gradient at the current step by the
  // adjoint recursion, then the new active sets from du - G / diag(Huu)
  // (written to box_act); returns whether any set changed
  auto update_sets = [&]() -> bool {
    T lam = 0;
    if (lane < NX)
      lam = (T)C.QN[lane] * ((T)x[(size_t)N * NX + lane] + (T)bdx[(size_t)N * NX + lane] -
                             (T)xr[(size_t)N * NX + lane]);
    bool changed = false;
    for (int k = N - 1; k >= 0; --k) {
      const size_t node = (size_t)uo + k;
      for (int e = lane; e < NX * NX; e += G) S.A[e / NX][e % NX] = (T)a.A[node * NX * NX + e];
      for (int e = lane; e < NX * NU; e += G) S.Bm[e / NU][e % NU] = (T)a.Bm[node * NX * NU + e];
      if (lane < NX) S.g[lane] = lam;
      __syncwarp(gm);
      if (lane < NU) {
        const T um = (T)u[(size_t)k * NU + lane];
        const T dum = (T)bdu[(size_t)k * NU + lane];
        T gr = (T)C.R[lane] * (um + dum - (T)ur[(size_t)k * NU + lane]);  // the cost's gradient
#pragma unroll
        for (int l = 0; l < NX; ++l) gr += S.Bm[l][lane] * S.g[l];
        const T v = dum - gr / (T)ka.box_gam[node * NU + lane];
        const signed char nw = v < -um ? -1 : (v > (T)ka.u_max - um ? 1 : 0);
        if (nw != ka.box_act[node * NU + lane]) {
          changed = true;
          ka.box_act[node * NU + lane] = nw;
        }
      }
      T ln = 0;
      if (lane < NX) {
        ln = (T)C.Q[lane] * ((T)x[(size_t)k * NX + lane] + (T)bdx[(size_t)k * NX + lane] -
                             (T)xr[(size_t)k * NX + lane]);
#pragma unroll
        for (int l = 0; l < NX; ++l) ln += S.A[l][lane] * S.g[l];
      }
      __syncwarp(gm);
      lam = ln;
    }
    return __any_sync(gm, changed);
  };

  // every du of the scratch step within 0 <= u + du <= u_max
  auto feasible = [&]() -> bool {
    bool ok = true;
    for (int e = lane; e < N * NU; e += G) {
      const float um = u[e], d = bdu[e];
      ok &= (d >= -um) && (d <= ka.u_max - um);
    }
    return __all_sync(gm, ok);
  };

  int st = finite ? RTN_OK : RTN_E_NONFINITE;
  if (st == RTN_OK && !BOX) {
    sweep();
    if (S.notpd) st = RTN_E_NOT_PD;
  } else if (BOX && st == RTN_OK) {
    // primal-dual active set: solve without bounds; while the step leaves
    // the box, update the sets and solve with the active inputs held at
    // their bounds, until the sets repeat (at most box_max_iter solves)
    for (int e = lane; e < N * NU; e += G) ka.box_act[(size_t)uo * NU + e] = 0;
    __syncwarp(gm);
    sweep();
    int its = 1;
    if (S.notpd) {
      st = RTN_E_NOT_PD;
    } else {
      forward(1, false);
      if (!feasible()) {
        for (;;) {
          const bool changed = update_sets();
          if (!changed && its > 1) break;
          if (its >= ka.box_max_iter) { st = RTN_E_NOT_CONVERGED; break; }
          sweep();
          ++its;
          if (S.notpd) { st = RTN_E_NOT_PD; break; }
          forward(1, false);
        }
      }
    }
    if (lane == 0) ka.box_iters[b] = its;
  }
  if (lane == 0 && a.status) a.status[b] = st;
  if (st != RTN_OK && st != RTN_E_NOT_CONVERGED) {
    // failed instance: zero step, iterate untouched, send the reference input
    if (a.dx)
      for (int e = lane; e < (N + 1) * NX; e += G) a.dx[(size_t)xo * NX + e] = 0.0f;
    if (a.du)
      for (int e = lane; e < N * NU; e += G) a.du[(size_t)uo * NU + e] = 0.0f;
    if (a.u0 && lane < NU) a.u0[(size_t)b * NU + lane] = ur[lane];
    return;
  }
  if constexpr (!BOX) forward(0, false);
  else forward(2, st == RTN_E_NOT_CONVERGED);
}

// WPB warps per block, 32 / G instances per warp (consecutive in the
// longest-first order, so the two halves of a warp mostly share N)
template <typename T, int WPB, bool BOX, bool CH64, int G>
__global__ void __launch_bounds__(WPB * 32, 5) qp_kernel(KArgs ka) {
  constexpr int GPW = 32 / G;
  __shared__ SlotOf<T, CH64> slots[WPB * GPW];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = warp * GPW + lane / G;
  const int slot = blockIdx.x * WPB * GPW + grp;
  if (slot >= ka.B) return;
  const int b = ka.order ? ka.order[slot] : slot;
  const unsigned gm = G == 32 ? 0xffffffffu : (0xffffu << (lane & 16));
  qp_instance<T, BOX, CH64, G>(ka, b, slots[grp], lane % G, gm);
}

// ---------------------------------------------------------------- latency mode
// One instance per block of QB threads, for batches small enough that a
// warp's sweep would run as one dependent chain with nothing to hide its
// latencies (one controller, N = 10: ~17k dependent warp instructions and a
// global-memory round trip or two per node, 38 us).  The instance's A, B,
// c, x, xref, u, uref are loaded into shared memory at once (coalesced,
// 268 floats per node), every product of a Riccati step is spread over the
// block, each output evaluated by one thread with the same expression in
// the same order as qp_instance (the results are those of the warp kernel
// bit for bit), and the gains stay in shared memory for the roll-out; the
// Cholesky of Huu stays on one thread, the solves on 14, and the part of
// the next P that needs no gains (Q + A'PA, q + A'g) is formed beside
// B'PA, off their path.  The unconstrained QP only (the box QP keeps the
// warp kernel).  One controller, N = 10: 31 -> ~24 us with 256 threads
// against 128.
constexpr int QB = 256;
constexpr int QB_NODE = NX * NX + NX * NU + NX + NX + NX + NU + NU;  // floats per node
constexpr size_t QB_SMEM_MAX = 160 * 1024;  // dynamic shared memory of the latency mode (N up to ~110)

// dynamic shared memory of qp_block_kernel for horizons up to n_max
template <typename T>
size_t qp_block_smem(int n_max) {
  const size_t f = ((size_t)QB_NODE * n_max + 2 * NX + 1) / 2 * 2 * sizeof(float);  // 8-byte aligned
  return f + (size_t)(NU * NX + NU) * n_max * sizeof(T);
}

template <typename T, bool CH64>
__global__ void __launch_bounds__(QB) qp_block_kernel(KArgs ka) {
  using TC = typename std::conditional<CH64, double, T>::type;
  __shared__ SlotOf<T, CH64> S;
  __shared__ __align__(16) T Pm[NX][16];  // P, row i
  __shared__ T pv[16], p2v[16];          // p and the next p
  extern __shared__ __align__(16) float qsm[];
  if ((int)blockIdx.x >= ka.B) return;
  const int tid = threadIdx.x;
  const int b = ka.order ? ka.order[blockIdx.x] : (int)blockIdx.x;
  const QpArgs& a = ka.a;
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
  // shared copies: A [N][13][13], B [N][13][4], c [N][13], x, xref [N + 1][13],
  // u, uref [N][4]; then the gains K [N][4][13], k [N][4]
  float* sA = qsm;
  float* sB = sA + (size_t)N * NX * NX;
  float* sc = sB + (size_t)N * NX * NU;
  float* sx = sc + (size_t)N * NX;
  float* sxr = sx + (size_t)(N + 1) * NX;
  float* su = sxr + (size_t)(N + 1) * NX;
  float* sur = su + (size_t)N * NU;
  T* sK = reinterpret_cast<T*>(qsm + ((size_t)QB_NODE * N + 2 * NX + 1) / 2 * 2);
  T* sk = sK + (size_t)N * NU * NX;
  {
    const size_t node0 = (size_t)uo;
    for (int e = tid; e < N * NX * NX; e += QB) sA[e] = a.A[node0 * NX * NX + e];
    for (int e = tid; e < N * NX * NU; e += QB) sB[e] = a.Bm[node0 * NX * NU + e];
    for (int e = tid; e < N * NX; e += QB) sc[e] = a.c[node0 * NX + e];
    for (int e = tid; e < (N + 1) * NX; e += QB) {
      sx[e] = x[e];
      sxr[e] = xr[e];
    }
    for (int e = tid; e < N * NU; e += QB) {
      su[e] = u[e];
      sur[e] = ur[e];
    }
  }

  // measured state
  const float x0m = tid < NX ? a.x0[(size_t)b * NX + tid] : 0.0f;
  const bool finite = __syncthreads_and(isfinite(x0m)) != 0;

  // ---------------- backward Riccati sweep
  for (int e = tid; e < NX * NX; e += QB) Pm[e / NX][e % NX] = (e / NX == e % NX) ? (T)C.QN[e / NX] : (T)0;
  if (tid < NX) pv[tid] = (T)C.QN[tid] * ((T)sx[(size_t)N * NX + tid] - (T)sxr[(size_t)N * NX + tid]);
  if (tid == 0) S.notpd = 0;
  __syncthreads();
  for (int k = N - 1; k >= 0 && finite; --k) {
    const size_t node = (size_t)uo + k;
    const float* Ak = sA + (size_t)k * NX * NX;  // A_k [l][j] at l * 13 + j
    const float* Bk = sB + (size_t)k * NX * NU;  // B_k [l][m] at l * 4 + m
    const float* ck = sc + (size_t)k * NX;
    // PA = P A (169), PB = P B (52), g = p + P c (13): row i, column cc
    for (int o = tid; o < NX * (NX + NU + 1); o += QB) {
      const int i = o / (NX + NU + 1), cc = o % (NX + NU + 1);
      if (cc < NX) {
        T s = 0;
#pragma unroll
        for (int l = 0; l < NX; ++l) s += Pm[i][l] * (T)Ak[l * NX + cc];
        S.PA[i][cc] = s;
      } else if (cc < NX + NU) {
        T s = 0;
#pragma unroll
        for (int l = 0; l < NX; ++l) s += Pm[i][l] * (T)Bk[l * NU + cc - NX];
        S.PB[i][cc - NX] = s;
      } else {
        T s = pv[i];
#pragma unroll
        for (int l = 0; l < NX; ++l) s += Pm[i][l] * (T)ck[l];
        S.g[i] = s;
      }
    }
    __syncthreads();
    // Hux = B'PA (52), Huu = R + B'PB (16), hu = r + B'g (4); beside them
    // the first terms of the next P and p: P2 = Q + A'PA (169), p2 = q + A'g
    // (13), finished with Hux'K and Hux'k once the gains are known
    for (int o = tid; o < NU * NX + NU * NU + NU + NX * NX + NX; o += QB) {
      T s = 0;
      if (o >= NU * NX + NU * NU + NU) {
        const int e = o - (NU * NX + NU * NU + NU);
        if (e < NX * NX) {
          const int i = e / NX, j = e % NX;
          s = (j == i) ? (T)C.Q[i] : (T)0;
#pragma unroll
          for (int l = 0; l < NX; ++l) s += (T)Ak[l * NX + i] * S.PA[l][j];
          S.P2[i][j] = s;
        } else {
          const int i = e - NX * NX;
          s = (T)C.Q[i] * ((T)sx[(size_t)k * NX + i] - (T)sxr[(size_t)k * NX + i]);
#pragma unroll
          for (int l = 0; l < NX; ++l) s += (T)Ak[l * NX + i] * S.g[l];
          p2v[i] = s;
        }
      } else if (o < NU * NX) {
        const int m = o / NX, j = o % NX;
#pragma unroll
        for (int l = 0; l < NX; ++l) s += (T)Bk[l * NU + m] * S.PA[l][j];
        S.Hux[m][j] = s;
      } else if (o < NU * NX + NU * NU) {
        const int e = o - NU * NX, m = e / NU, n = e % NU;
        s = (m == n) ? (T)C.R[m] : (T)0;
#pragma unroll
        for (int l = 0; l < NX; ++l) s += (T)Bk[l * NU + m] * S.PB[l][n];
        S.Huu[e] = s;
      } else {
        const int m = o - NU * NX - NU * NU;
        s = (T)C.R[m] * ((T)su[(size_t)k * NU + m] - (T)sur[(size_t)k * NU + m]);
#pragma unroll
        for (int l = 0; l < NX; ++l) s += (T)Bk[l * NU + m] * S.g[l];
        S.hu[m] = s;
      }
    }
    __syncthreads();
    // Cholesky of Huu by one thread (one reciprocal square root per pivot)
    if (tid == 0) {
      TC L[NU][NU];
      bool pd = true;
#pragma unroll
      for (int j = 0; j < NU; ++j) {
        TC s = (TC)S.Huu[j * NU + j];
#pragma unroll
        for (int q = 0; q < j; ++q) s -= L[j][q] * L[j][q];
        pd &= (s > (TC)0);
        TC inv;
        if constexpr (sizeof(TC) == 4) inv = rsqrtf(fmaxf(s, 1e-30f));
        else inv = rsqrt(fmax(s, 1e-300));
        L[j][j] = s * inv;
        S.Linvt[j] = (T)inv;
#pragma unroll
        for (int i = j + 1; i < NU; ++i) {
          TC v = (TC)S.Huu[i * NU + j];
#pragma unroll
          for (int q = 0; q < j; ++q) v -= L[i][q] * L[j][q];
          L[i][j] = v * inv;
        }
      }
#pragma unroll
      for (int i = 0; i < NU; ++i)
#pragma unroll
        for (int j = 0; j < NU; ++j) S.Lt[i * NU + j] = (j < i) ? (T)L[i][j] : (T)0;
      if (!pd) S.notpd = 1;
    }
    __syncthreads();
    // [K | k] = -Huu^{-1} [Hux | hu]: right-hand side `tid` (13 = hu); the
    // gains to global memory and to the shared copies of the roll-out
    if (tid < NX + 1) {
      T y[NU];
#pragma unroll
      for (int i = 0; i < NU; ++i) {
        T v = (tid < NX) ? S.Hux[i][tid] : S.hu[i];
#pragma unroll
        for (int q = 0; q < i; ++q) v -= S.Lt[i * NU + q] * y[q];
        y[i] = v * S.Linvt[i];
      }
#pragma unroll
      for (int i = NU - 1; i >= 0; --i) {
        T v = y[i];
#pragma unroll
        for (int q = i + 1; q < NU; ++q) v -= S.Lt[q * NU + i] * y[q];
        y[i] = v * S.Linvt[i];
      }
#pragma unroll
      for (int i = 0; i < NU; ++i) {
        const T g = -y[i];
        if (tid < NX) {
          S.K[i][tid] = g;
          sK[((size_t)k * NU + i) * NX + tid] = g;
          Kg[node * NU * NX + i * NX + tid] = g;
        } else {
          S.k[i] = g;
          sk[(size_t)k * NU + i] = g;
          kg[node * NU + i] = g;
        }
      }
    }
    __syncthreads();
    // P2 += Hux'K (169), p2 += Hux'k (13)
    for (int o = tid; o < NX * NX + NX; o += QB) {
      if (o < NX * NX) {
        const int i = o / NX, j = o % NX;
        T s = S.P2[i][j];
#pragma unroll
        for (int m = 0; m < NU; ++m) s += S.Hux[m][i] * S.K[m][j];
        S.P2[i][j] = s;
      } else {
        const int i = o - NX * NX;
        T s = p2v[i];
#pragma unroll
        for (int m = 0; m < NU; ++m) s += S.Hux[m][i] * S.k[m];
        p2v[i] = s;
      }
    }
    __syncthreads();
    // P = (P2 + P2') / 2, p = p2
    for (int o = tid; o < NX * NX; o += QB) {
      const int i = o / NX, j = o % NX;
      Pm[i][j] = (T)0.5 * (S.P2[i][j] + S.P2[j][i]);
    }
    if (tid < NX) pv[tid] = p2v[tid];
    __syncthreads();
    (void)node;
  }
  int st = finite ? RTN_OK : RTN_E_NONFINITE;
  if (st == RTN_OK && S.notpd) st = RTN_E_NOT_PD;
  if (tid == 0 && a.status) a.status[b] = st;
  if (st != RTN_OK) {
    // failed instance: zero step, iterate untouched, send the reference input
    if (a.dx)
      for (int e = tid; e < (N + 1) * NX; e += QB) a.dx[(size_t)xo * NX + e] = 0.0f;
    if (a.du)
      for (int e = tid; e < N * NU; e += QB) a.du[(size_t)uo * NU + e] = 0.0f;
    if (a.u0 && tid < NU) a.u0[(size_t)b * NU + tid] = ur[tid];
    return;
  }

  // ---------------- forward roll-out from dx_0 = x0 - x_0: du = K dx + k,
  // the step to a.dx / a.du, the iterate update (and shift), u0; every
  // operand from the shared copies (the iterate's old values among them, so
  // the in-place update of x, u needs no ordering)
  float* xw = a.x + (size_t)xo * NX;
  float* uw = a.u + (size_t)uo * NU;
  if (tid < NX) S.dx[tid] = (T)x0m - (T)sx[tid];
  __syncthreads();
  if (tid < NX) {
    if (a.dx) a.dx[(size_t)xo * NX + tid] = (float)S.dx[tid];
    if (a.update && !a.shift) xw[tid] = (float)((T)sx[tid] + S.dx[tid]);
  }
  for (int k = 0; k < N; ++k) {
    const size_t node = (size_t)uo + k;
    if (tid < NU) {
      const T* Kr = sK + ((size_t)k * NU + tid) * NX;
      T s = sk[(size_t)k * NU + tid];
#pragma unroll
      for (int j = 0; j < NX; ++j) s += Kr[j] * S.dx[j];
      S.du[tid] = s;
    }
    __syncthreads();
    T dxn = 0;
    if (tid < NX) {
      const float* Ar = sA + (size_t)k * NX * NX + tid * NX;
      const float* Br = sB + (size_t)k * NX * NU + tid * NU;
      T s = (T)sc[(size_t)k * NX + tid];
#pragma unroll
      for (int j = 0; j < NX; ++j) s += (T)Ar[j] * S.dx[j];
#pragma unroll
      for (int j = 0; j < NU; ++j) s += (T)Br[j] * S.du[j];
      dxn = s;
    }
    if (tid < NU) {
      T unew = (T)su[(size_t)k * NU + tid] + S.du[tid];
      if (a.du) a.du[node * NU + tid] = (float)S.du[tid];
      if (k == 0 && a.u0) {
        float v = (float)unew;
        a.u0[(size_t)b * NU + tid] = fminf(fmaxf(v, 0.0f), ka.u_max);
      }
      if (a.update) {
        if (a.shift) {
          if (k >= 1) uw[(size_t)(k - 1) * NU + tid] = (float)unew;
          if (k == N - 1) uw[(size_t)k * NU + tid] = (float)unew;
        } else {
          uw[(size_t)k * NU + tid] = (float)unew;
        }
      }
    }
    if (tid < NX) {
      if (a.dx) a.dx[(size_t)(xo + k + 1) * NX + tid] = (float)dxn;
      if (a.update) {
        T xnew = (T)sx[(size_t)(k + 1) * NX + tid] + dxn;
        if (a.shift) {
          xw[(size_t)k * NX + tid] = (float)xnew;
          if (k == N - 1) xw[(size_t)(k + 1) * NX + tid] = (float)xnew;
        } else {
          xw[(size_t)(k + 1) * NX + tid] = (float)xnew;
        }
      }
    }
    __syncthreads();
    if (tid < NX) S.dx[tid] = dxn;
    __syncthreads();
  }
}

// ---------------------------------------------------------------- fused
// The RK4 linearisation (a2) and the QP (a3 + a4) of every instance in one
// persistent launch.  Warps first take units of 32 (node, column) RK4
// threads from an atomic ticket, nodes in longest-horizon-first instance
// order, and count the columns they finish per instance; when the units
// are exhausted they take instances (same order) and run each one's QP once
// all of its columns are counted.  Every unit a QP waits for was taken by a
// running warp, so the waits end; they are bounded all the same.  The
// latency-bound sweeps of the long instances overlap the issue-bound RK4
// work of the short ones.
constexpr int FQ_WPB = 4;

struct FusedArgs {
  KArgs ka;
  QuadParams P;
  const float *x, *u, *fD, *JD;
  const int *node_inst, *rk_nodes;
  const float* dt;
  int n_nodes;
  int* counters;  // [0] RK4 unit ticket, [1] QP ticket, [2] warps finished, [3 + b] columns of instance b finished
  int* err;       // device status word (RTN_E_TIMEOUT)
  long long wait_cycles;
  int stall;      // fault injection: every QP waits for one column more than exists
};

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__global__ void __launch_bounds__(FQ_WPB * 32, 4) lin_qp_kernel(FusedArgs fa) {
  __shared__ SlotOf<float, false> slots[FQ_WPB];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long total = (long long)fa.n_nodes * NZ;
  const long long n_units = (total + 31) / 32;
  int* rk_next = fa.counters;
  int* qp_next = fa.counters + 1;
  int* finished = fa.counters + 2;
  int* done = fa.counters + 3;
  const QpArgs& a = fa.ka.a;
  for (;;) {
    int unit = 0;
    if (lane == 0) unit = atomicAdd(rk_next, 1);
    unit = __shfl_sync(0xffffffffu, unit, 0);
    if (unit >= n_units) break;
    const long long tid = (long long)unit * 32 + lane;
    int b = -1;
    if (tid < total) {
      const int n = fa.rk_nodes[tid / NZ];
      rk4_column<NO>(fa.P, fa.x, fa.u, fa.fD, fa.JD, nullptr, fa.node_inst, fa.dt, n, (int)(tid % NZ), const_cast<float*>(a.A),
                     const_cast<float*>(a.Bm), const_cast<float*>(a.c));
      b = fa.node_inst[n];
    }
    // publish the finished columns: one atomic per instance in the unit
    __threadfence();
    const unsigned grp = __match_any_sync(0xffffffffu, b);
    if (b >= 0 && lane == __ffs(grp) - 1) atomicAdd(done + b, __popc(grp));
  }
  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(qp_next, 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= fa.ka.B) break;
    const int b = fa.ka.order[t];
    const int need = fa.ka.N[b] * NZ + fa.stall;
    int ok = 1;
    if (lane == 0) {
      if (ld_acquire(done + b) < need) {
        const long long t0 = clock64();
        while (ld_acquire(done + b) < need) {
          if (clock64() - t0 > fa.wait_cycles) {
            ok = 0;
            atomicExch(fa.err, (int)RTN_E_TIMEOUT);
            break;
          }
          __nanosleep(100);
        }
      }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __threadfence();
    if (!ok) {
      // the instance's linearisation never completed: no step, reference input
      if (lane == 0 && a.status) a.status[b] = RTN_E_TIMEOUT;
      if (a.u0 && lane < NU) {
        const int ur0 = (a.uref_stride > 0 ? b * a.uref_stride : fa.ka.uoff[b]) + (a.t_dev ? *a.t_dev : 0);
        a.u0[(size_t)b * NU + lane] = a.uref[(size_t)ur0 * NU + lane];
      }
      continue;
    }
    qp_instance<float, false, false, 32>(fa.ka, b, slots[warp], lane, 0xffffffffu);
  }
  // the last warp to finish (every other warp has taken its last ticket and
  // finished its work) returns the counters to zero for the next launch
  int last = 0;
  if (lane == 0) {
    __threadfence();
    last = atomicAdd(finished, 1) == (int)(gridDim.x * FQ_WPB) - 1;
  }
  if (__shfl_sync(0xffffffffu, last, 0)) {
    __threadfence();
    for (int e = lane; e < fa.ka.B; e += 32) done[e] = 0;
    if (lane == 0) {
      *rk_next = 0;
      *qp_next = 0;
      *finished = 0;
    }
    __threadfence();
  }
}

template <typename T, int WPB, bool CH64 = false, int G = 32>
cudaError_t launch(const KArgs& ka, cudaStream_t s) {
  const int per_block = WPB * (32 / G);
  const int grid = (ka.B + per_block - 1) / per_block;
  if (ka.box) qp_kernel<T, WPB, true, CH64, G><<<grid, WPB * 32, 0, s>>>(ka);
  else qp_kernel<T, WPB, false, CH64, G><<<grid, WPB * 32, 0, s>>>(ka);
  return cudaGetLastError();
}


KArgs make_kargs(rtn_ctx* ctx, const QpArgs& a) {
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
  ka.box = ctx->opt.box_qp;
  ka.box_max_iter = ctx->opt.box_max_iter;
  ka.box_dx = ctx->box_dx;
  ka.box_du = ctx->box_du;
  ka.box_gam = ctx->box_gam;
  ka.box_act = ctx->box_act;
  ka.box_iters = ctx->box_iters;
  return ka;
}

}  // namespace

// lanes per instance of the FP32 sweeps (rtn_options.qp_group; 0: automatic).
// Measured on 1024..16384 instances (N = 20, and N in 10..50): the box QP
// is faster on whole warps at every size (its active-set loop diverges
// between the instances of a warp); the sweep with the FP64 factorisation on
// half warps at every size (its FP64 instructions serve two instances); the
// FP32 sweep on half warps once the batch's work exceeds what the resident
// warps finish in the longest horizon's chain (sum N_b > resident x N_max),
// on whole warps below (a half-warp step is ~1.2x slower unloaded)
// Batches of at most one instance per SM run one block per instance (QB
// threads: the latency of one controller's QP).
int qp_group(const rtn_ctx* ctx) {
  if (ctx->opt.qp_group == QB)  // one block per instance: no bounds, horizons whose data fit shared memory
    return ctx->opt.box_qp || qp_block_smem<double>(ctx->lay.N_max) > QB_SMEM_MAX ? 32 : QB;
  if (ctx->opt.qp_group) return ctx->opt.qp_group;
  if (ctx->opt.box_qp) return 32;
  static int resident = 0, sms = 0;          // warps of qp_kernel resident on the GPU, SMs
  if (!resident) {
    int dev = 0, n = 148, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, qp_kernel<float, 4, false, false, 32>, 128, 0);
    sms = std::max(1, n);
    resident = std::max(1, sms * std::max(occ, 1) * 4);
  }
  if (ctx->B <= sms && qp_block_smem<double>(ctx->lay.N_max) <= QB_SMEM_MAX) return QB;
  if (ctx->opt.riccati_f64 == 2) return 16;
  return (long long)ctx->lay.n_nodes > (long long)resident * ctx->lay.N_max ? 16 : 32;
}

template <typename T, bool CH64>
cudaError_t launch_block(const KArgs& ka, int n_max, cudaStream_t s) {
  const size_t smem = qp_block_smem<T>(n_max);
  cudaError_t e = cudaFuncSetAttribute(qp_block_kernel<T, CH64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  qp_block_kernel<T, CH64><<<ka.B, QB, smem, s>>>(ka);
  return cudaGetLastError();
}

cudaError_t qp_solve(rtn_ctx* ctx, const QpArgs& a) {
  const KArgs ka = make_kargs(ctx, a);
  if (qp_group(ctx) == QB) {  // one block per instance (no input bounds)
    const int n_max = ctx->lay.N_max;
    if (ctx->opt.riccati_f64 == 1) return launch_block<double, false>(ka, n_max, ctx->stream);
    if (ctx->opt.riccati_f64 == 2) return launch_block<float, true>(ka, n_max, ctx->stream);
    return launch_block<float, false>(ka, n_max, ctx->stream);
  }
  if (ctx->opt.riccati_f64 == 1) return launch<double, 2>(ka, ctx->stream);
  const bool g16 = qp_group(ctx) == 16;
  if (ctx->opt.riccati_f64 == 2)
    return g16 ? launch<float, 4, true, 16>(ka, ctx->stream) : launch<float, 4, true, 32>(ka, ctx->stream);
  return g16 ? launch<float, 4, false, 16>(ka, ctx->stream) : launch<float, 4, false, 32>(ka, ctx->stream);
}

bool lin_qp_fusable(const rtn_ctx* ctx) {
  return ctx->opt.fused_qp && !ctx->di && ctx->n_out == NO && !ctx->opt.second_order && !ctx->opt.box_qp &&
         ctx->opt.riccati_f64 == 0;
}

cudaError_t lin_qp_solve(rtn_ctx* ctx, const QpArgs& a, const float* fD, const float* JD) {
  FusedArgs fa;
  fa.ka = make_kargs(ctx, a);
  fa.P = ctx->quad;
  fa.x = a.x;
  fa.u = a.u;
  fa.fD = fD;
  fa.JD = JD;
  fa.node_inst = ctx->lay.node_inst;
  fa.rk_nodes = ctx->lay.rk_nodes;
  fa.dt = ctx->lay.dt;
  fa.n_nodes = ctx->lay.n_nodes;
  fa.counters = ctx->lay.counters;
  fa.err = ctx->net.tc.err;
  fa.wait_cycles = ctx->net.tc.wait_cycles > 0 ? ctx->net.tc.wait_cycles : 4000000000LL;
  fa.stall = ctx->net.tc.inject_stall ? 1 : 0;
  if (!fa.err) return cudaErrorInvalidValue;
  static int grid = 0;
  if (!grid) {
    int dev = 0, sms = 148, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lin_qp_kernel, FQ_WPB * 32, 0);
    grid = sms * std::max(occ, 1);
  }
  // the counters are zero from create and returned to zero by each launch's last warp
  lin_qp_kernel<<<grid, FQ_WPB * 32, 0, ctx->stream>>>(fa);
  return cudaGetLastError();
}

}  // namespace rtn
