// plant.cu -- (a5) the simulated plant of a closed loop, in FP64.
//
// The plant integrates the true dynamics f_F + f_res over one control
// interval with nsub RK4 sub-steps (u held), then renormalises the attitude
// quaternion.  f_F is the nominal model of Sec. V (Eq. 6); f_res is one of
//   - none,
//   - body drag  -R diag(0.3, 0.3, 0.1) R' v - 0.01 |v| v  (world frame),
//   - the residual network evaluated exactly (no local model): 3 outputs
//     added to dv/dt, or 6 (the full residual of Eq. 7, rows 3-5 added to
//     dw/dt; in the state order [p, q, v, w] row r lands on component 7 + r).
// One thread per instance; the network variant reads an FP64 weight copy.
#include "rtn_internal.cuh"

namespace rtn {
namespace {

constexpr int PLANT_MAX_W = 64;

struct PlantNet {
  int n_layers;
  int widths[12];
  const double* P;  // per layer: W [out][in] then b [out]
};

__device__ void qmul_d(const double* a, const double* b, double* r) {
  r[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  r[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
  r[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
  r[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

// rotate v by q (q v q^*) or by its conjugate
__device__ void rotate_d(const double* q, const double* v, double* o, bool conj) {
  double qq[4] = {q[0], conj ? -q[1] : q[1], conj ? -q[2] : q[2], conj ? -q[3] : q[3]};
  double qc[4] = {qq[0], -qq[1], -qq[2], -qq[3]};
  double pv[4] = {0.0, v[0], v[1], v[2]}, t[4], r[4];
  qmul_d(qq, pv, t);
  qmul_d(t, qc, r);
  o[0] = r[1]; o[1] = r[2]; o[2] = r[3];
}

__device__ void dyn_true(const rtn_quad& P, int kind, const PlantNet& net, const double* x,
                         const double* u, double* xd) {
  xd[0] = x[7]; xd[1] = x[8]; xd[2] = x[9];
  double w[4] = {0.0, 0.5 * x[10], 0.5 * x[11], 0.5 * x[12]};
  qmul_d(x + 3, w, xd + 3);
  double T = u[0] + u[1] + u[2] + u[3];
  double tb[3] = {0.0, 0.0, T}, a[3];
  rotate_d(x + 3, tb, a, false);
  xd[7] = a[0] / P.mass;
  xd[8] = a[1] / P.mass;
  xd[9] = a[2] / P.mass - P.g;
  double d = P.arm / sqrt(2.0);
  double tx = d * (u[2] + u[3] - u[0] - u[1]);
  double ty = d * (u[1] + u[2] - u[0] - u[3]);
  double tz = P.c_tau * (u[1] + u[3] - u[0] - u[2]);
  double wx = x[10], wy = x[11], wz = x[12];
  xd[10] = (tx - (P.Jz - P.Jy) * wy * wz) / P.Jx;
  xd[11] = (ty - (P.Jx - P.Jz) * wz * wx) / P.Jy;
  xd[12] = (tz - (P.Jy - P.Jx) * wx * wy) / P.Jz;
  if (kind == RTN_PLANT_DRAG) {
    double vb[3], db[3], dw[3];
    rotate_d(x + 3, x + 7, vb, true);
    db[0] = 0.3 * vb[0]; db[1] = 0.3 * vb[1]; db[2] = 0.1 * vb[2];
    rotate_d(x + 3, db, dw, false);
    double nv = sqrt(x[7] * x[7] + x[8] * x[8] + x[9] * x[9]);
    for (int i = 0; i < 3; ++i) xd[7 + i] += -dw[i] - 0.01 * nv * x[7 + i];
  } else if (kind == RTN_PLANT_MLP) {
    double a0[PLANT_MAX_W], a1[PLANT_MAX_W];
    for (int i = 0; i < NX; ++i) a0[i] = x[i];
    for (int i = 0; i < NU; ++i) a0[NX + i] = u[i];
    const double* p = net.P;
    for (int l = 0; l < net.n_layers; ++l) {
      int fi = net.widths[l], fo = net.widths[l + 1];
      const double* Wl = p;
      const double* bl = p + fo * fi;
      for (int i = 0; i < fo; ++i) {
        double s = bl[i];
        for (int j = 0; j < fi; ++j) s += Wl[i * fi + j] * a0[j];
        a1[i] = (l < net.n_layers - 1) ? tanh(s) : s;
      }
      for (int i = 0; i < fo; ++i) a0[i] = a1[i];
      p += fo * fi + fo;
    }
    for (int i = 0; i < net.widths[net.n_layers]; ++i) xd[7 + i] += a0[i];
  }
}

__global__ void plant_kernel(rtn_quad P, int kind, PlantNet net, int B,
                             const double* __restrict__ dt, const double* x,
                             const float* __restrict__ u, double* xn, int nsub,
                             float* __restrict__ xf) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double s[NX], k1[NX], k2[NX], k3[NX], k4[NX], t[NX], uu[NU];
  for (int i = 0; i < NX; ++i) s[i] = x[(size_t)b * NX + i];
  for (int i = 0; i < NU; ++i) uu[i] = (double)u[(size_t)b * NU + i];
  double h = dt[b] / nsub;
  for (int it = 0; it < nsub; ++it) {
    dyn_true(P, kind, net, s, uu, k1);
    for (int i = 0; i < NX; ++i) t[i] = s[i] + 0.5 * h * k1[i];
    dyn_true(P, kind, net, t, uu, k2);
    for (int i = 0; i < NX; ++i) t[i] = s[i] + 0.5 * h * k2[i];
    dyn_true(P, kind, net, t, uu, k3);
    for (int i = 0; i < NX; ++i) t[i] = s[i] + h * k3[i];
    dyn_true(P, kind, net, t, uu, k4);
    for (int i = 0; i < NX; ++i) s[i] += h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
  }
  double nq = sqrt(s[3] * s[3] + s[4] * s[4] + s[5] * s[5] + s[6] * s[6]);
  for (int i = 3; i < 7; ++i) s[i] /= nq;
  for (int i = 0; i < NX; ++i) {
    xn[(size_t)b * NX + i] = s[i];
    if (xf) xf[(size_t)b * NX + i] = (float)s[i];
  }
}

}  // namespace

cudaError_t plant_step(rtn_ctx* ctx, int kind, const double* x, const float* u, double* xn,
                       int nsub, float* x_f32) {
  PlantNet pn{};
  if (kind == RTN_PLANT_MLP) {
    if (!ctx->has_mlp || ctx->net.n_layers > 11 || ctx->net.h_max > PLANT_MAX_W)
      return cudaErrorNotSupported;
    pn.n_layers = ctx->net.n_layers;
    for (int l = 0; l <= pn.n_layers; ++l) pn.widths[l] = ctx->net.widths[l];
    pn.P = ctx->net.P64;
  }
  plant_kernel<<<(ctx->B + 127) / 128, 128, 0, ctx->stream>>>(ctx->quad64, kind, pn, ctx->B,
                                                              ctx->lay.dt64, x, u, xn, nsub, x_f32);
  return cudaGetLastError();
}

}  // namespace rtn
