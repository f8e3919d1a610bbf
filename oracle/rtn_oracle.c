/*
 * rtn_oracle.c -- plain, slow, FP64 CPU oracle for the Real-time Neural MPC
 * hot path (Salzmann et al., "Real-time Neural MPC", RA-L 2023).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code;
 * only the tests, the package's smoke check and the benchmark's CPU-baseline
 * arm use it.  It shares no code, header, table or constant generator with the
 * CUDA path.
 *
 * Every routine is the textbook definition written out with plain loops, in
 * the order the paper states the method:
 *   - MLP residual f_D and its input Jacobian J_D (Sec. III-A, Eq. 4):
 *     forward-mode and, as an independent cross-check, reverse-mode.
 *   - Nominal quadrotor model f_F (Sec. V, Eq. 6) with the rotor layout of
 *     Fig. 3, and its analytic Jacobian.
 *   - RK4 phi (Sec. II, Eq. 1) of f_F + f_D* where f_D* is the first-order
 *     local model of Eq. 4, with the sensitivities A_k, B_k of the continuity
 *     condition (Eq. 2) obtained by propagating d(stage)/d[x;u].
 *   - The QP of Sec. III-A with the quadratic tracking cost of Sec. V, solved
 *     by the textbook Riccati recursion, plus a dense KKT solve used as a pin;
 *     with the thrust bounds of Sec. V, by a primal-dual active-set method
 *     whose subproblems are masked Riccati recursions.
 *   - One RTI step (Sec. III-B): linearise, solve, update the iterate, shift.
 *   - Plant step, closed loop, drag residual, and MLP training (MSE + Adam,
 *     Sec. VI).
 *
 * Sign conventions and readings where the paper is silent:
 *   - state x = [p(3), q(4) w-first, v(3), omega(3)], u = [T0..T3];
 *   - rotor body positions (Fig. 3, X layout, d = arm/sqrt2):
 *     r0=(+d,-d) r1=(-d,-d) r2=(-d,+d) r3=(+d,+d); rotors 0,2 spin CCW,
 *     1,3 CW seen from +z, so tau_z = c_tau(-T0+T1-T2+T3);
 *   - q (.) v is the literal product q v q^* (not normalised);
 *   - the residual network's 3 outputs are a world-frame acceleration added
 *     to dv/dt;
 *   - cost 1/2|x-x_r|_Q^2 + 1/2|u-u_r|_R^2 per stage, terminal 1/2|x_N-x_r|_QN^2.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NX 13
#define NU 4
#define NZ 17

typedef struct {
  double mass, Jx, Jy, Jz, arm, c_tau, u_max, g;
} orc_quad;

/* ------------------------------------------------------------------ MLP --- */
/* Parameters packed per layer l: W_l [w[l+1]][w[l]] row-major, then b_l. */

static int mlp_max_width(int nl, const int* w) {
  int m = 0;
  for (int l = 0; l <= nl; ++l) if (w[l] > m) m = w[l];
  return m;
}

/* value of the network: hidden layers tanh, last layer linear */
void orc_mlp_forward(int nl, const int* w, const double* P, const double* z, double* out) {
  int hm = mlp_max_width(nl, w);
  double* a = (double*)malloc(sizeof(double) * hm);
  double* t = (double*)malloc(sizeof(double) * hm);
  for (int i = 0; i < w[0]; ++i) a[i] = z[i];
  const double* p = P;
  for (int l = 0; l < nl; ++l) {
    int fi = w[l], fo = w[l + 1];
    const double* W = p;
    const double* b = p + (size_t)fo * fi;
    for (int i = 0; i < fo; ++i) {
      double s = b[i];
      for (int j = 0; j < fi; ++j) s += W[(size_t)i * fi + j] * a[j];
      t[i] = (l < nl - 1) ? tanh(s) : s;
    }
    for (int i = 0; i < fo; ++i) a[i] = t[i];
    p += (size_t)fo * fi + fo;
  }
  for (int i = 0; i < w[nl]; ++i) out[i] = a[i];
  free(a);
  free(t);
}

/* forward-mode: propagate the value and the n_in tangent directions together
 * (the seed is the identity), J[out][in] */
void orc_mlp_fwd_jac(int nl, const int* w, const double* P, const double* z, double* f,
                     double* J) {
  int hm = mlp_max_width(nl, w), nin = w[0];
  double* a = (double*)malloc(sizeof(double) * hm);
  double* T = (double*)malloc(sizeof(double) * hm * nin);
  double* a2 = (double*)malloc(sizeof(double) * hm);
  double* T2 = (double*)malloc(sizeof(double) * hm * nin);
  for (int i = 0; i < nin; ++i) {
    a[i] = z[i];
    for (int j = 0; j < nin; ++j) T[i * nin + j] = (i == j) ? 1.0 : 0.0;
  }
  const double* p = P;
  for (int l = 0; l < nl; ++l) {
    int fi = w[l], fo = w[l + 1];
    const double* W = p;
    const double* b = p + (size_t)fo * fi;
    for (int i = 0; i < fo; ++i) {
      double s = b[i];
      for (int k = 0; k < fi; ++k) s += W[(size_t)i * fi + k] * a[k];
      for (int j = 0; j < nin; ++j) {
        double tj = 0.0;
        for (int k = 0; k < fi; ++k) tj += W[(size_t)i * fi + k] * T[k * nin + j];
        T2[i * nin + j] = tj;
      }
      if (l < nl - 1) {
        double th = tanh(s), d = 1.0 - th * th;
        a2[i] = th;
        for (int j = 0; j < nin; ++j) T2[i * nin + j] *= d;
      } else {
        a2[i] = s;
      }
    }
    for (int i = 0; i < fo; ++i) {
      a[i] = a2[i];
      for (int j = 0; j < nin; ++j) T[i * nin + j] = T2[i * nin + j];
    }
    p += (size_t)fo * fi + fo;
  }
  for (int i = 0; i < w[nl]; ++i) {
    f[i] = a[i];
    for (int j = 0; j < nin; ++j) J[i * nin + j] = T[i * nin + j];
  }
  free(a); free(T); free(a2); free(T2);
}

/* second order (the H_D of Eq. 4): forward-over-forward, carrying per unit
 * the value a, the tangents t_j = da/dz_j and the second derivatives
 * s_jm = d^2 a / dz_j dz_m through every layer.  With the pre-activation
 * y = W a + b (tangents W t, second derivatives W s) and a = tanh(y):
 *   t_j = tanh'(y) (W t)_j,
 *   s_jm = tanh'(y) (W s)_jm + tanh''(y) (W t)_j (W t)_m,
 * tanh' = 1 - a^2, tanh'' = -2 a (1 - a^2); the last layer is linear.
 * f [nout], J [nout][nin], H [nout][nin][nin]. */
void orc_mlp_fwd_hess(int nl, const int* w, const double* P, const double* z, double* f, double* J,
                      double* H) {
  int hm = mlp_max_width(nl, w), nin = w[0], n2 = nin * nin;
  double* a = (double*)malloc(sizeof(double) * hm);
  double* T = (double*)malloc(sizeof(double) * hm * nin);
  double* S = (double*)malloc(sizeof(double) * hm * n2);
  double* a2 = (double*)malloc(sizeof(double) * hm);
  double* T2 = (double*)malloc(sizeof(double) * hm * nin);
  double* S2 = (double*)malloc(sizeof(double) * hm * n2);
  for (int i = 0; i < nin; ++i) {
    a[i] = z[i];
    for (int j = 0; j < nin; ++j) T[i * nin + j] = (i == j) ? 1.0 : 0.0;
    for (int j = 0; j < n2; ++j) S[i * n2 + j] = 0.0;
  }
  const double* p = P;
  for (int l = 0; l < nl; ++l) {
    int fi = w[l], fo = w[l + 1];
    const double* W = p;
    const double* b = p + (size_t)fo * fi;
    for (int i = 0; i < fo; ++i) {
      double y = b[i];
      for (int k = 0; k < fi; ++k) y += W[(size_t)i * fi + k] * a[k];
      for (int j = 0; j < nin; ++j) {
        double t = 0.0;
        for (int k = 0; k < fi; ++k) t += W[(size_t)i * fi + k] * T[k * nin + j];
        T2[i * nin + j] = t;
      }
      for (int j = 0; j < n2; ++j) {
        double v = 0.0;
        for (int k = 0; k < fi; ++k) v += W[(size_t)i * fi + k] * S[(size_t)k * n2 + j];
        S2[(size_t)i * n2 + j] = v;
      }
      if (l < nl - 1) {
        double th = tanh(y), d1 = 1.0 - th * th, d2 = -2.0 * th * d1;
        a2[i] = th;
        for (int j = 0; j < nin; ++j)
          for (int m = 0; m < nin; ++m)
            S2[(size_t)i * n2 + j * nin + m] =
                d1 * S2[(size_t)i * n2 + j * nin + m] + d2 * T2[i * nin + j] * T2[i * nin + m];
        for (int j = 0; j < nin; ++j) T2[i * nin + j] *= d1;
      } else {
        a2[i] = y;
      }
    }
    for (int i = 0; i < fo; ++i) {
      a[i] = a2[i];
      for (int j = 0; j < nin; ++j) T[i * nin + j] = T2[i * nin + j];
      for (int j = 0; j < n2; ++j) S[(size_t)i * n2 + j] = S2[(size_t)i * n2 + j];
    }
    p += (size_t)fo * fi + fo;
  }
  for (int i = 0; i < w[nl]; ++i) {
    f[i] = a[i];
    for (int j = 0; j < nin; ++j) J[i * nin + j] = T[i * nin + j];
    for (int j = 0; j < n2; ++j) H[(size_t)i * n2 + j] = S[(size_t)i * n2 + j];
  }
  free(a); free(T); free(S); free(a2); free(T2); free(S2);
}

/* reverse-mode cross-check: forward pass storing activations, then one
 * adjoint sweep per output row */
void orc_mlp_rev_jac(int nl, const int* w, const double* P, const double* z, double* J) {
  int hm = mlp_max_width(nl, w), nin = w[0], nout = w[nl];
  double* acts = (double*)malloc(sizeof(double) * hm * (nl + 1));
  double* g = (double*)malloc(sizeof(double) * hm);
  double* g2 = (double*)malloc(sizeof(double) * hm);
  const double** Ws = (const double**)malloc(sizeof(double*) * nl);
  for (int i = 0; i < nin; ++i) acts[i] = z[i];
  const double* p = P;
  for (int l = 0; l < nl; ++l) {
    int fi = w[l], fo = w[l + 1];
    Ws[l] = p;
    const double* b = p + (size_t)fo * fi;
    for (int i = 0; i < fo; ++i) {
      double s = b[i];
      for (int k = 0; k < fi; ++k) s += p[(size_t)i * fi + k] * acts[l * hm + k];
      acts[(l + 1) * hm + i] = (l < nl - 1) ? tanh(s) : s;
    }
    p += (size_t)fo * fi + fo;
  }
  for (int r = 0; r < nout; ++r) {
    for (int i = 0; i < nout; ++i) g[i] = (i == r) ? 1.0 : 0.0;
    for (int l = nl - 1; l >= 0; --l) {
      int fi = w[l], fo = w[l + 1];
      if (l < nl - 1)
        for (int i = 0; i < fo; ++i) {
          double th = acts[(l + 1) * hm + i];
          g[i] *= 1.0 - th * th;
        }
      for (int k = 0; k < fi; ++k) {
        double s = 0.0;
        for (int i = 0; i < fo; ++i) s += Ws[l][(size_t)i * fi + k] * g[i];
        g2[k] = s;
      }
      for (int k = 0; k < fi; ++k) g[k] = g2[k];
    }
    for (int j = 0; j < nin; ++j) J[r * nin + j] = g[j];
  }
  free(acts); free(g); free(g2); free(Ws);
}

/* ------------------------------------------------------------ quadrotor --- */

static void qmul(const double* a, const double* b, double* r) {
  r[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  r[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
  r[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
  r[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

/* q (.) v = q (0,v) q^*   (Sec. V, notation) */
void orc_qrot(const double* q, const double* v, double* out) {
  double pv[4] = {0.0, v[0], v[1], v[2]}, t[4], r[4];
  double qc[4] = {q[0], -q[1], -q[2], -q[3]};
  qmul(q, pv, t);
  qmul(t, qc, r);
  out[0] = r[1]; out[1] = r[2]; out[2] = r[3];
}

/* body torque from the four rotor thrusts, Fig. 3 reading */
static void rotor_torque(const orc_quad* Qd, const double* u, double* tau) {
  double d = Qd->arm / sqrt(2.0);
  tau[0] = d * (-u[0] - u[1] + u[2] + u[3]);
  tau[1] = d * (-u[0] + u[1] + u[2] - u[3]);
  tau[2] = Qd->c_tau * (-u[0] + u[1] - u[2] + u[3]);
}

/* nominal model f_F, Eq. 6 */
void orc_quad_f(const orc_quad* Qd, const double* x, const double* u, double* xd) {
  const double* q = x + 3;
  const double* v = x + 7;
  const double* om = x + 10;
  xd[0] = v[0]; xd[1] = v[1]; xd[2] = v[2];
  double po[4] = {0.0, om[0] / 2.0, om[1] / 2.0, om[2] / 2.0};
  qmul(q, po, xd + 3);
  double TB[3] = {0.0, 0.0, u[0] + u[1] + u[2] + u[3]}, a[3];
  orc_qrot(q, TB, a);
  xd[7] = a[0] / Qd->mass;
  xd[8] = a[1] / Qd->mass;
  xd[9] = a[2] / Qd->mass - Qd->g;
  double J[3] = {Qd->Jx, Qd->Jy, Qd->Jz}, tau[3], Jw[3], c[3];
  rotor_torque(Qd, u, tau);
  for (int i = 0; i < 3; ++i) Jw[i] = J[i] * om[i];
  c[0] = om[1] * Jw[2] - om[2] * Jw[1];
  c[1] = om[2] * Jw[0] - om[0] * Jw[2];
  c[2] = om[0] * Jw[1] - om[1] * Jw[0];
  for (int i = 0; i < 3; ++i) xd[10 + i] = (tau[i] - c[i]) / J[i];
}

/* analytic Jacobian of f_F with respect to [x; u]: D[13][17] */
void orc_quad_dfdz(const orc_quad* Qd, const double* x, const double* u, double* D) {
  memset(D, 0, sizeof(double) * NX * NZ);
#define DD(r, c) D[(r) * NZ + (c)]
  const double qw = x[3], qx = x[4], qy = x[5], qz = x[6];
  const double wx = x[10], wy = x[11], wz = x[12];
  /* dp/dt = v */
  for (int i = 0; i < 3; ++i) DD(i, 7 + i) = 1.0;
  /* dq/dt = 1/2 q (x) (0, w) */
  double Wq[4][4] = {{0, -wx, -wy, -wz}, {wx, 0, wz, -wy}, {wy, -wz, 0, wx}, {wz, wy, -wx, 0}};
  double Qw[4][3] = {{-qx, -qy, -qz}, {qw, -qz, qy}, {qz, qw, -qx}, {-qy, qx, qw}};
  for (int i = 0; i < 4; ++i) {
    for (int j = 0; j < 4; ++j) DD(3 + i, 3 + j) = 0.5 * Wq[i][j];
    for (int j = 0; j < 3; ++j) DD(3 + i, 10 + j) = 0.5 * Qw[i][j];
  }
  /* dv/dt = (T/m) q (.) e_z - g e_z */
  double T = u[0] + u[1] + u[2] + u[3], m = Qd->mass;
  double r[3] = {2 * (qx * qz + qw * qy), 2 * (qy * qz - qw * qx), qw * qw - qx * qx - qy * qy + qz * qz};
  double dr[3][4] = {{2 * qy, 2 * qz, 2 * qw, 2 * qx},
                     {-2 * qx, -2 * qw, 2 * qz, 2 * qy},
                     {2 * qw, -2 * qx, -2 * qy, 2 * qz}};
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 4; ++j) DD(7 + i, 3 + j) = T / m * dr[i][j];
    for (int j = 0; j < 4; ++j) DD(7 + i, 13 + j) = r[i] / m;
  }
  /* dw/dt = J^-1 (tau - w x J w) */
  double Jx = Qd->Jx, Jy = Qd->Jy, Jz = Qd->Jz;
  DD(10, 11) = -(Jz - Jy) * wz / Jx; DD(10, 12) = -(Jz - Jy) * wy / Jx;
  DD(11, 10) = -(Jx - Jz) * wz / Jy; DD(11, 12) = -(Jx - Jz) * wx / Jy;
  DD(12, 10) = -(Jy - Jx) * wy / Jz; DD(12, 11) = -(Jy - Jx) * wx / Jz;
  double d = Qd->arm / sqrt(2.0), c = Qd->c_tau;
  double tx[4] = {-d, -d, d, d}, ty[4] = {-d, d, d, -d}, tz[4] = {-c, c, -c, c};
  for (int j = 0; j < 4; ++j) {
    DD(10, 13 + j) = tx[j] / Jx;
    DD(11, 13 + j) = ty[j] / Jy;
    DD(12, 13 + j) = tz[j] / Jz;
  }
#undef DD
}

/* f_F + f_D* where f_D* is the local model of Eq. 4 around (xk, uk),
 * fbar + J dz (+ 1/2 dz' H_r dz with H != NULL, the second-order model),
 * dz = [x - xk; u - uk].  With no = 3 outputs the residual is a linear
 * acceleration added to dv/dt; with no = 6 it is the full residual of Eq. 7,
 * [0; 0; f_theta; f_psi]: rows 0-2 added to dv/dt, rows 3-5 (angular
 * acceleration) to dw/dt.  In the state order [p, q, v, w] row r lands on
 * component 7 + r in both cases. */
static void f_local(const orc_quad* Qd, const double* x, const double* u, const double* xk,
                    const double* uk, int no, const double* fbar, const double* J, const double* H,
                    double* xd) {
  orc_quad_f(Qd, x, u, xd);
  if (!fbar) return;
  double dz[NZ];
  for (int i = 0; i < NX; ++i) dz[i] = x[i] - xk[i];
  for (int i = 0; i < NU; ++i) dz[NX + i] = u[i] - uk[i];
  for (int r = 0; r < no; ++r) {
    double s = fbar[r];
    for (int j = 0; j < NZ; ++j) s += J[r * NZ + j] * dz[j];
    if (H)
      for (int j = 0; j < NZ; ++j)
        for (int m = 0; m < NZ; ++m) s += 0.5 * dz[j] * H[(r * NZ + j) * NZ + m] * dz[m];
    xd[7 + r] += s;
  }
}

/* RK4 (u held) of f_F + f_D*, with the sensitivity S = d(stage)/d[x;u]
 * (13 x 17) propagated through the four stages:
 *   phi = x + dt/6 (k1 + 2 k2 + 2 k3 + k4),  A = dphi/dx,  B = dphi/du.
 * fbar/J may be NULL (nominal model only). */
void orc_rk4_lin_n(const orc_quad* Qd, const double* x, const double* u, int no, const double* fbar,
                   const double* J, const double* H, double dt, double* phi, double* A, double* B) {
  double k[4][NX], dk[4][NX * NZ], xs[NX], S[NX * NZ], D[NX * NZ];
  double cst[4] = {0.0, 0.5, 0.5, 1.0};
  for (int s = 0; s < 4; ++s) {
    for (int i = 0; i < NX; ++i) xs[i] = x[i] + (s ? cst[s] * dt * k[s - 1][i] : 0.0);
    for (int i = 0; i < NX; ++i)
      for (int j = 0; j < NZ; ++j)
        S[i * NZ + j] = ((i == j) ? 1.0 : 0.0) + (s ? cst[s] * dt * dk[s - 1][i * NZ + j] : 0.0);
    f_local(Qd, xs, u, x, u, no, fbar, J, H, k[s]);
    orc_quad_dfdz(Qd, xs, u, D);
    /* the local model's gradient at the stage point: J_r (+ H_r dz) */
    if (fbar)
      for (int r = 0; r < no; ++r)
        for (int j = 0; j < NZ; ++j) {
          double g = J[r * NZ + j];
          if (H)
            for (int m = 0; m < NX; ++m) g += H[(r * NZ + j) * NZ + m] * (xs[m] - x[m]);
          D[(7 + r) * NZ + j] += g;
        }
    /* d k_s / d[x;u] = Dx * S + Du * [0 I] */
    for (int i = 0; i < NX; ++i)
      for (int j = 0; j < NZ; ++j) {
        double sum = (j >= NX) ? D[i * NZ + j] : 0.0;
        for (int l = 0; l < NX; ++l) sum += D[i * NZ + l] * S[l * NZ + j];
        dk[s][i * NZ + j] = sum;
      }
  }
  for (int i = 0; i < NX; ++i) {
    phi[i] = x[i] + dt / 6.0 * (k[0][i] + 2.0 * k[1][i] + 2.0 * k[2][i] + k[3][i]);
    for (int j = 0; j < NZ; ++j) {
      double v = ((i == j) ? 1.0 : 0.0) +
                 dt / 6.0 * (dk[0][i * NZ + j] + 2.0 * dk[1][i * NZ + j] + 2.0 * dk[2][i * NZ + j] +
                             dk[3][i * NZ + j]);
      if (j < NX) A[i * NX + j] = v;
      else B[i * NU + (j - NX)] = v;
    }
  }
}

/* the 3-output residual (linear acceleration only) */
void orc_rk4_lin_h(const orc_quad* Qd, const double* x, const double* u, const double* fbar,
                   const double* J, const double* H, double dt, double* phi, double* A, double* B) {
  orc_rk4_lin_n(Qd, x, u, 3, fbar, J, H, dt, phi, A, B);
}

void orc_rk4_lin(const orc_quad* Qd, const double* x, const double* u, const double* fbar,
                 const double* J, double dt, double* phi, double* A, double* B) {
  orc_rk4_lin_n(Qd, x, u, 3, fbar, J, NULL, dt, phi, A, B);
}

/* drag residual used as the ground-truth aerodynamics:
 * a = -R(q) diag(0.3,0.3,0.1) R(q)^T v - 0.01 |v| v  (world-frame accel.) */
void orc_drag(const double* x, double* a) {
  const double* q = x + 3;
  const double* v = x + 7;
  double qc[4] = {q[0], -q[1], -q[2], -q[3]}, vb[3], db[3];
  orc_qrot(qc, v, vb);
  db[0] = 0.3 * vb[0]; db[1] = 0.3 * vb[1]; db[2] = 0.1 * vb[2];
  orc_qrot(q, db, a);
  double nv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  for (int i = 0; i < 3; ++i) a[i] = -a[i] - 0.01 * nv * v[i];
}

/* true dynamics of the plant: f_F + residual; kind 0 none, 1 drag, 2 MLP
 * (3 outputs added to dv/dt, or 6: the full residual of Eq. 7, rows 3-5
 * added to dw/dt) */
static void f_true(const orc_quad* Qd, int kind, int nl, const int* w, const double* P,
                   const double* x, const double* u, double* xd) {
  orc_quad_f(Qd, x, u, xd);
  double r[6] = {0, 0, 0, 0, 0, 0};
  const int no = (kind == 2 && nl > 0) ? w[nl] : 3;
  if (kind == 1) orc_drag(x, r);
  if (kind == 2) {
    double z[NZ];
    for (int i = 0; i < NX; ++i) z[i] = x[i];
    for (int i = 0; i < NU; ++i) z[NX + i] = u[i];
    orc_mlp_forward(nl, w, P, z, r);
  }
  for (int i = 0; i < no; ++i) xd[7 + i] += r[i];
}

/* plain RK4 step of the true dynamics (no renormalisation) */
void orc_rk4_true(const orc_quad* Qd, int kind, int nl, const int* w, const double* P,
                  const double* x, const double* u, double dt, double* xn) {
  double k1[NX], k2[NX], k3[NX], k4[NX], t[NX];
  f_true(Qd, kind, nl, w, P, x, u, k1);
  for (int i = 0; i < NX; ++i) t[i] = x[i] + 0.5 * dt * k1[i];
  f_true(Qd, kind, nl, w, P, t, u, k2);
  for (int i = 0; i < NX; ++i) t[i] = x[i] + 0.5 * dt * k2[i];
  f_true(Qd, kind, nl, w, P, t, u, k3);
  for (int i = 0; i < NX; ++i) t[i] = x[i] + dt * k3[i];
  f_true(Qd, kind, nl, w, P, t, u, k4);
  for (int i = 0; i < NX; ++i) xn[i] = x[i] + dt / 6.0 * (k1[i] + 2 * k2[i] + 2 * k3[i] + k4[i]);
}

/* plant: nsub RK4 sub-steps of dt/nsub, then q <- q/|q| */
void orc_plant_step(const orc_quad* Qd, int kind, int nl, const int* w, const double* P,
                    const double* x, const double* u, double dt, int nsub, double* xn) {
  double a[NX], b[NX];
  memcpy(a, x, sizeof(a));
  for (int s = 0; s < nsub; ++s) {
    orc_rk4_true(Qd, kind, nl, w, P, a, u, dt / nsub, b);
    memcpy(a, b, sizeof(a));
  }
  double n = sqrt(a[3] * a[3] + a[4] * a[4] + a[5] * a[5] + a[6] * a[6]);
  for (int i = 3; i < 7; ++i) a[i] /= n;
  memcpy(xn, a, sizeof(a));
}

/* -------------------------------------------------------------- linear algebra */

/* Cholesky of a small SPD matrix (lower), returns 0 if not positive definite */
static int chol(int n, const double* M, double* L) {
  memset(L, 0, sizeof(double) * n * n);
  for (int j = 0; j < n; ++j) {
    double s = M[j * n + j];
    for (int k = 0; k < j; ++k) s -= L[j * n + k] * L[j * n + k];
    if (!(s > 0.0)) return 0;
    L[j * n + j] = sqrt(s);
    for (int i = j + 1; i < n; ++i) {
      double t = M[i * n + j];
      for (int k = 0; k < j; ++k) t -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = t / L[j * n + j];
    }
  }
  return 1;
}

/* solve (L L^T) X = Bm for ncol right-hand sides stored column-major-ish:
 * Bm[n][ncol] row-major, overwritten by X */
static void chol_solve(int n, const double* L, int ncol, double* Bm) {
  for (int c = 0; c < ncol; ++c) {
    for (int i = 0; i < n; ++i) {
      double s = Bm[i * ncol + c];
      for (int k = 0; k < i; ++k) s -= L[i * n + k] * Bm[k * ncol + c];
      Bm[i * ncol + c] = s / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double s = Bm[i * ncol + c];
      for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * Bm[k * ncol + c];
      Bm[i * ncol + c] = s / L[i * n + i];
    }
  }
}

/* ------------------------------------------------------------------- QP --- */
/*
 * One linear-quadratic subproblem (Sec. III-A; cost of Sec. V):
 *   min sum_k 1/2 dx'Q dx + q'dx + 1/2 du'R du + r'du  + 1/2 dxN'QN dxN + pN'dxN
 *   s.t. dx_0 = x0meas - x_0,  dx_{k+1} = A_k dx_k + B_k du_k + c_k    (Eq. 2)
 * with q_k = Q(x_k - xr_k), r_k = R(u_k - ur_k), pN = QN(x_N - xr_N).
 * Solved by the Riccati recursion (backward), then the forward roll-out.
 * Generic sizes nx, nu so that a scalar special case can be checked.
 * Q, R, QN are diagonal (vectors).  Returns 0 on success, 4 if not PD.
 */
/* Core of the recursion.  With fixed != NULL, input i of node k is held at
 * du_k[i] = aval[k*nu+i] wherever fixed[k*nu+i] != 0 and the others are
 * optimised (an equality-constrained LQ subproblem of the box-constrained QP
 * below): at each node the free inputs solve Huu_ff du_f = -(hu_f + Huu_fA a)
 * - Hux_f dx, the fixed rows of K are zero and of k the held values, and the
 * cost-to-go update uses the full Hux.  gam (optional) receives diag(Huu). */
static int riccati_core(int nx, int nu, int N, const double* A, const double* Bm, const double* c,
                        const double* x, const double* u, const double* xr, const double* ur,
                        const double* Q, const double* R, const double* QN, const double* x0m,
                        const int* fixed, const double* aval, double* dx, double* du,
                        double* Kout, double* kout, double* gam) {
  int ok = 1;
  double* P = (double*)calloc(nx * nx, sizeof(double));
  double* p = (double*)calloc(nx, sizeof(double));
  double* K = (double*)calloc((size_t)N * nu * nx, sizeof(double));
  double* kf = (double*)calloc((size_t)N * nu, sizeof(double));
  double* PA = (double*)malloc(sizeof(double) * nx * nx);
  double* PB = (double*)malloc(sizeof(double) * nx * nu);
  double* Huu = (double*)malloc(sizeof(double) * nu * nu);
  double* Hux = (double*)malloc(sizeof(double) * nu * nx);
  double* Lc = (double*)malloc(sizeof(double) * nu * nu);
  double* g = (double*)malloc(sizeof(double) * nx);
  double* hu = (double*)malloc(sizeof(double) * nu);
  double* P2 = (double*)malloc(sizeof(double) * nx * nx);
  double* p2 = (double*)malloc(sizeof(double) * nx);
  double* rhs = (double*)malloc(sizeof(double) * nu * (nx + 1));
  for (int i = 0; i < nx; ++i) {
    P[i * nx + i] = QN[i];
    p[i] = QN[i] * (x[(size_t)N * nx + i] - xr[(size_t)N * nx + i]);
  }
  for (int k = N - 1; k >= 0; --k) {
    const double* Ak = A + (size_t)k * nx * nx;
    const double* Bk = Bm + (size_t)k * nx * nu;
    const double* ck = c + (size_t)k * nx;
    for (int i = 0; i < nx; ++i) {
      for (int j = 0; j < nx; ++j) {
        double s = 0;
        for (int l = 0; l < nx; ++l) s += P[i * nx + l] * Ak[l * nx + j];
        PA[i * nx + j] = s;
      }
      for (int j = 0; j < nu; ++j) {
        double s = 0;
        for (int l = 0; l < nx; ++l) s += P[i * nx + l] * Bk[l * nu + j];
        PB[i * nu + j] = s;
      }
      double s = p[i];
      for (int l = 0; l < nx; ++l) s += P[i * nx + l] * ck[l];
      g[i] = s; /* p + P c */
    }
    for (int i = 0; i < nu; ++i) {
      for (int j = 0; j < nu; ++j) {
        double s = (i == j) ? R[i] : 0.0;
        for (int l = 0; l < nx; ++l) s += Bk[l * nu + i] * PB[l * nu + j];
        Huu[i * nu + j] = s;
      }
      for (int j = 0; j < nx; ++j) {
        double s = 0;
        for (int l = 0; l < nx; ++l) s += Bk[l * nu + i] * PA[l * nx + j];
        Hux[i * nx + j] = s;
      }
      double s = R[i] * (u[(size_t)k * nu + i] - ur[(size_t)k * nu + i]);
      for (int l = 0; l < nx; ++l) s += Bk[l * nu + i] * g[l];
      hu[i] = s;
    }
    if (gam)
      for (int i = 0; i < nu; ++i) gam[(size_t)k * nu + i] = Huu[i * nu + i];
    /* [K | k] = -Huu^{-1} [Hux | hu]  (fixed inputs: identity rows/columns,
     * zero rows of Hux, right-hand side -a; coupling moved to the free rows) */
    for (int i = 0; i < nu; ++i) {
      const int fi = fixed && fixed[(size_t)k * nu + i];
      for (int j = 0; j < nx; ++j) rhs[i * (nx + 1) + j] = fi ? 0.0 : Hux[i * nx + j];
      double h = hu[i];
      if (fi) {
        h = -aval[(size_t)k * nu + i];
      } else if (fixed) {
        for (int m = 0; m < nu; ++m)
          if (fixed[(size_t)k * nu + m]) h += Huu[i * nu + m] * aval[(size_t)k * nu + m];
      }
      rhs[i * (nx + 1) + nx] = h;
    }
    if (fixed) {
      for (int i = 0; i < nu; ++i)
        for (int m = 0; m < nu; ++m)
          if (fixed[(size_t)k * nu + i] || fixed[(size_t)k * nu + m])
            Huu[i * nu + m] = (i == m) ? 1.0 : 0.0;
    }
    if (!chol(nu, Huu, Lc)) { ok = 0; break; }
    chol_solve(nu, Lc, nx + 1, rhs);
    double* Kk = K + (size_t)k * nu * nx;
    double* kk = kf + (size_t)k * nu;
    for (int i = 0; i < nu; ++i) {
      for (int j = 0; j < nx; ++j) Kk[i * nx + j] = -rhs[i * (nx + 1) + j];
      kk[i] = -rhs[i * (nx + 1) + nx];
    }
    /* P <- Q + A'PA + Hux'K ;  p <- q + A'(p + Pc) + Hux'k */
    for (int i = 0; i < nx; ++i) {
      for (int j = 0; j < nx; ++j) {
        double s = (i == j) ? Q[i] : 0.0;
        for (int l = 0; l < nx; ++l) s += Ak[l * nx + i] * PA[l * nx + j];
        for (int l = 0; l < nu; ++l) s += Hux[l * nx + i] * Kk[l * nx + j];
        P2[i * nx + j] = s;
      }
      double s = Q[i] * (x[(size_t)k * nx + i] - xr[(size_t)k * nx + i]);
      for (int l = 0; l < nx; ++l) s += Ak[l * nx + i] * g[l];
      for (int l = 0; l < nu; ++l) s += Hux[l * nx + i] * kk[l];
      p2[i] = s;
    }
    for (int i = 0; i < nx; ++i) {
      for (int j = 0; j < nx; ++j) P[i * nx + j] = 0.5 * (P2[i * nx + j] + P2[j * nx + i]);
      p[i] = p2[i];
    }
  }
  if (ok) {
    for (int i = 0; i < nx; ++i) dx[i] = x0m[i] - x[i];
    for (int k = 0; k < N; ++k) {
      const double* Ak = A + (size_t)k * nx * nx;
      const double* Bk = Bm + (size_t)k * nx * nu;
      const double* ck = c + (size_t)k * nx;
      const double* Kk = K + (size_t)k * nu * nx;
      const double* kk = kf + (size_t)k * nu;
      double* dxk = dx + (size_t)k * nx;
      double* duk = du + (size_t)k * nu;
      for (int i = 0; i < nu; ++i) {
        double s = kk[i];
        for (int j = 0; j < nx; ++j) s += Kk[i * nx + j] * dxk[j];
        duk[i] = s;
      }
      for (int i = 0; i < nx; ++i) {
        double s = ck[i];
        for (int j = 0; j < nx; ++j) s += Ak[i * nx + j] * dxk[j];
        for (int j = 0; j < nu; ++j) s += Bk[i * nu + j] * duk[j];
        dxk[nx + i] = s;
      }
    }
    if (Kout) memcpy(Kout, K, sizeof(double) * N * nu * nx);
    if (kout) memcpy(kout, kf, sizeof(double) * N * nu);
  }
  free(P); free(p); free(K); free(kf); free(PA); free(PB); free(Huu); free(Hux); free(Lc);
  free(g); free(hu); free(P2); free(p2); free(rhs);
  return ok ? 0 : 4;
}

int orc_riccati(int nx, int nu, int N, const double* A, const double* Bm, const double* c,
                const double* x, const double* u, const double* xr, const double* ur,
                const double* Q, const double* R, const double* QN, const double* x0m,
                double* dx, double* du, double* Kout, double* kout) {
  return riccati_core(nx, nu, N, A, Bm, c, x, u, xr, ur, Q, R, QN, x0m, NULL, NULL, dx, du, Kout,
                      kout, NULL);
}

/* Gradient of the QP's cost with respect to every du_k along a trajectory
 * (dx, du) that satisfies the dynamics, by the adjoint recursion:
 *   lam_N = QN (x_N + dx_N - xr_N),
 *   G_k = R (u_k + du_k - ur_k) + B_k' lam_{k+1},
 *   lam_k = Q (x_k + dx_k - xr_k) + A_k' lam_{k+1}. */
static void qp_gradient(int nx, int nu, int N, const double* A, const double* Bm, const double* x,
                        const double* u, const double* xr, const double* ur, const double* Q,
                        const double* R, const double* QN, const double* dx, const double* du,
                        double* G) {
  double* lam = (double*)malloc(sizeof(double) * nx);
  double* l2 = (double*)malloc(sizeof(double) * nx);
  for (int i = 0; i < nx; ++i)
    lam[i] = QN[i] * (x[(size_t)N * nx + i] + dx[(size_t)N * nx + i] - xr[(size_t)N * nx + i]);
  for (int k = N - 1; k >= 0; --k) {
    const double* Ak = A + (size_t)k * nx * nx;
    const double* Bk = Bm + (size_t)k * nx * nu;
    for (int i = 0; i < nu; ++i) {
      double s = R[i] * (u[(size_t)k * nu + i] + du[(size_t)k * nu + i] - ur[(size_t)k * nu + i]);
      for (int l = 0; l < nx; ++l) s += Bk[l * nu + i] * lam[l];
      G[(size_t)k * nu + i] = s;
    }
    for (int i = 0; i < nx; ++i) {
      double s = Q[i] * (x[(size_t)k * nx + i] + dx[(size_t)k * nx + i] - xr[(size_t)k * nx + i]);
      for (int l = 0; l < nx; ++l) s += Ak[l * nx + i] * lam[l];
      l2[i] = s;
    }
    memcpy(lam, l2, sizeof(double) * nx);
  }
  free(lam); free(l2);
}

/*
 * The same QP with box constraints on the inputs, lb_k <= du_k <= ub_k (the
 * thrust bounds 0 <= u_k + du_k <= u_max of Sec. V), by a primal-dual active
 * set method on the Riccati structure:
 *   1. solve without bounds; if feasible, that is the solution;
 *   2. otherwise, with G the gradient of the cost at the current solution and
 *      gamma = diag(Huu) per node, the new active sets are
 *        lower = {du - G/gamma < lb},  upper = {du - G/gamma > ub};
 *      hold those inputs at their bounds and solve the equality-constrained
 *      subproblem (riccati_core with a mask); repeat until the sets repeat,
 *      which is then a KKT point: free inputs inside the box with zero
 *      gradient, held inputs with multipliers of the right sign.
 * At most max_iter subproblems are solved.  Returns 0 on convergence, 4 if a
 * Huu is not positive definite, 8 if the sets did not settle within max_iter
 * (then du is the last solution clamped to the box and dx its roll-out).
 * *iters receives the number of subproblems solved.
 */
int orc_box_qp(int nx, int nu, int N, const double* A, const double* Bm, const double* c,
               const double* x, const double* u, const double* xr, const double* ur,
               const double* Q, const double* R, const double* QN, const double* x0m,
               const double* lb, const double* ub, int max_iter, double* dx, double* du,
               int* iters) {
  const size_t n = (size_t)N * nu;
  int* fixed = (int*)calloc(n, sizeof(int));
  int* nfix = (int*)calloc(n, sizeof(int));
  double* aval = (double*)calloc(n, sizeof(double));
  double* gam = (double*)malloc(sizeof(double) * n);
  double* G = (double*)malloc(sizeof(double) * n);
  int st = riccati_core(nx, nu, N, A, Bm, c, x, u, xr, ur, Q, R, QN, x0m, NULL, NULL, dx, du, NULL,
                        NULL, gam);
  int it = 1, done = 0;
  if (st == 0) {
    done = 1;
    for (size_t i = 0; i < n; ++i)
      if (du[i] < lb[i] || du[i] > ub[i]) done = 0;
  }
  while (st == 0 && !done) {
    qp_gradient(nx, nu, N, A, Bm, x, u, xr, ur, Q, R, QN, dx, du, G);
    int changed = 0;
    for (size_t i = 0; i < n; ++i) {
      const double v = du[i] - G[i] / gam[i];
      nfix[i] = v < lb[i] ? -1 : (v > ub[i] ? 1 : 0);
      if (nfix[i] != fixed[i]) changed = 1;
    }
    if (!changed && it > 1) { done = 1; break; }
    if (it >= max_iter) {
      /* not settled: the last solution clamped to the box, rolled out */
      for (size_t i = 0; i < n; ++i) du[i] = du[i] < lb[i] ? lb[i] : (du[i] > ub[i] ? ub[i] : du[i]);
      for (int i = 0; i < nx; ++i) dx[i] = x0m[i] - x[i];
      for (int k = 0; k < N; ++k) {
        const double* Ak = A + (size_t)k * nx * nx;
        const double* Bk = Bm + (size_t)k * nx * nu;
        for (int i = 0; i < nx; ++i) {
          double s = c[(size_t)k * nx + i];
          for (int j = 0; j < nx; ++j) s += Ak[i * nx + j] * dx[(size_t)k * nx + j];
          for (int j = 0; j < nu; ++j) s += Bk[i * nu + j] * du[(size_t)k * nu + j];
          dx[(size_t)(k + 1) * nx + i] = s;
        }
      }
      st = 8;
      break;
    }
    for (size_t i = 0; i < n; ++i) {
      fixed[i] = nfix[i];
      aval[i] = nfix[i] < 0 ? lb[i] : (nfix[i] > 0 ? ub[i] : 0.0);
    }
    st = riccati_core(nx, nu, N, A, Bm, c, x, u, xr, ur, Q, R, QN, x0m, fixed, aval, dx, du, NULL,
                      NULL, gam);
    ++it;
  }
  if (iters) *iters = it;
  free(fixed); free(nfix); free(aval); free(gam); free(G);
  return st;
}

/* dense KKT solve of the same QP (LU with partial pivoting), used only as an
 * independent check of the Riccati recursion on tiny horizons */
int orc_kkt_dense(int nx, int nu, int N, const double* A, const double* Bm, const double* c,
                  const double* x, const double* u, const double* xr, const double* ur,
                  const double* Q, const double* R, const double* QN, const double* x0m,
                  double* dx, double* du) {
  int nxv = (N + 1) * nx, nuv = N * nu, nv = nxv + nuv, ne = (N + 1) * nx, n = nv + ne;
  double* M = (double*)calloc((size_t)n * n, sizeof(double));
  double* b = (double*)calloc(n, sizeof(double));
#define M_(i, j) M[(size_t)(i) * n + (j)]
  /* Hessian and gradient */
  for (int k = 0; k <= N; ++k)
    for (int i = 0; i < nx; ++i) {
      int vi = k * nx + i;
      double qq = (k < N) ? Q[i] : QN[i];
      M_(vi, vi) = qq;
      b[vi] = -qq * (x[k * nx + i] - xr[k * nx + i]);
    }
  for (int k = 0; k < N; ++k)
    for (int i = 0; i < nu; ++i) {
      int vi = nxv + k * nu + i;
      M_(vi, vi) = R[i];
      b[vi] = -R[i] * (u[k * nu + i] - ur[k * nu + i]);
    }
  /* equality constraints  C w = d */
  for (int i = 0; i < nx; ++i) {
    int r = nv + i;
    M_(r, i) = 1.0; M_(i, r) = 1.0;
    b[r] = x0m[i] - x[i];
  }
  for (int k = 0; k < N; ++k)
    for (int i = 0; i < nx; ++i) {
      int r = nv + (k + 1) * nx + i;
      /* dx_{k+1} - A dx_k - B du_k = c */
      M_(r, (k + 1) * nx + i) = 1.0; M_((k + 1) * nx + i, r) = 1.0;
      for (int j = 0; j < nx; ++j) {
        M_(r, k * nx + j) = -A[(size_t)k * nx * nx + i * nx + j];
        M_(k * nx + j, r) = -A[(size_t)k * nx * nx + i * nx + j];
      }
      for (int j = 0; j < nu; ++j) {
        M_(r, nxv + k * nu + j) = -Bm[(size_t)k * nx * nu + i * nu + j];
        M_(nxv + k * nu + j, r) = -Bm[(size_t)k * nx * nu + i * nu + j];
      }
      b[r] = c[k * nx + i];
    }
  /* Gaussian elimination with partial pivoting */
  int ok = 1;
  for (int col = 0; col < n && ok; ++col) {
    int piv = col;
    double best = fabs(M_(col, col));
    for (int r = col + 1; r < n; ++r)
      if (fabs(M_(r, col)) > best) { best = fabs(M_(r, col)); piv = r; }
    if (best == 0.0) { ok = 0; break; }
    if (piv != col) {
      for (int j = 0; j < n; ++j) { double t = M_(col, j); M_(col, j) = M_(piv, j); M_(piv, j) = t; }
      double t = b[col]; b[col] = b[piv]; b[piv] = t;
    }
    for (int r = col + 1; r < n; ++r) {
      double f = M_(r, col) / M_(col, col);
      if (f == 0.0) continue;
      for (int j = col; j < n; ++j) M_(r, j) -= f * M_(col, j);
      b[r] -= f * b[col];
    }
  }
  if (ok) {
    for (int i = n - 1; i >= 0; --i) {
      double s = b[i];
      for (int j = i + 1; j < n; ++j) s -= M_(i, j) * b[j];
      b[i] = s / M_(i, i);
    }
    memcpy(dx, b, sizeof(double) * nxv);
    memcpy(du, b + nxv, sizeof(double) * nuv);
  }
#undef M_
  free(M); free(b);
  return ok ? 0 : 1;
}

/* ------------------------------------------------------------- batched --- */

static void offsets(int B, const int* N, size_t* xo, size_t* uo) {
  size_t a = 0, c = 0;
  for (int b = 0; b < B; ++b) { xo[b] = a; uo[b] = c; a += N[b] + 1; c += N[b]; }
}

/* Linearise every shooting node (data-driven preparation + QP preparation,
 * Sec. III-B): fD[node][no], JD[node][no][17] (no = 3 or 6 network outputs),
 * A[node][13][13], B[node][13][4],
 * c[node][13] = phi_k - x_{k+1}.  nl = 0 means nominal model only. */
/* second != 0: the second-order local model (H_D from orc_mlp_fwd_hess,
 * written to HD [n][3][17][17] when HD != NULL) */
static void linearize_core(const orc_quad* Qd, int nl, const int* w, const double* P, int B,
                           const int* N, const double* dt, const double* x, const double* u,
                           double* fD, double* JD, double* HD, double* A, double* Bm, double* c,
                           int second) {
  size_t* xo = (size_t*)malloc(sizeof(size_t) * B);
  size_t* uo = (size_t*)malloc(sizeof(size_t) * B);
  offsets(B, N, xo, uo);
#pragma omp parallel for schedule(dynamic)
  for (int b = 0; b < B; ++b) {
    const int no = nl > 0 ? w[nl] : 3;
    double* H = (double*)malloc(sizeof(double) * 6 * NZ * NZ);
    for (int k = 0; k < N[b]; ++k) {
      size_t n = uo[b] + k;
      const double* xk = x + (xo[b] + k) * NX;
      const double* uk = u + n * NU;
      double z[NZ], f[6], J[6 * NZ], phi[NX];
      for (int i = 0; i < NX; ++i) z[i] = xk[i];
      for (int i = 0; i < NU; ++i) z[NX + i] = uk[i];
      if (nl > 0 && second) orc_mlp_fwd_hess(nl, w, P, z, f, J, H);
      else if (nl > 0) orc_mlp_fwd_jac(nl, w, P, z, f, J);
      else { memset(f, 0, sizeof(f)); memset(J, 0, sizeof(J)); }
      orc_rk4_lin_n(Qd, xk, uk, no, nl > 0 ? f : NULL, nl > 0 ? J : NULL, (nl > 0 && second) ? H : NULL,
                    dt[b], phi, A + n * NX * NX, Bm + n * NX * NU);
      for (int i = 0; i < NX; ++i) c[n * NX + i] = phi[i] - xk[NX + i];
      if (fD) memcpy(fD + n * no, f, sizeof(double) * no);
      if (JD) memcpy(JD + n * no * NZ, J, sizeof(double) * no * NZ);
      if (HD && second) memcpy(HD + n * no * NZ * NZ, H, sizeof(double) * no * NZ * NZ);
    }
    free(H);
  }
  free(xo); free(uo);
}

void orc_linearize(const orc_quad* Qd, int nl, const int* w, const double* P, int B,
                   const int* N, const double* dt, const double* x, const double* u, double* fD,
                   double* JD, double* A, double* Bm, double* c) {
  linearize_core(Qd, nl, w, P, B, N, dt, x, u, fD, JD, NULL, A, Bm, c, 0);
}

/* the same with the second-order local model of Eq. 4 (HD may be NULL) */
void orc_linearize2(const orc_quad* Qd, int nl, const int* w, const double* P, int B,
                    const int* N, const double* dt, const double* x, const double* u, double* fD,
                    double* JD, double* HD, double* A, double* Bm, double* c) {
  linearize_core(Qd, nl, w, P, B, N, dt, x, u, fD, JD, HD, A, Bm, c, 1);
}

/* One real-time iteration for every instance (Sec. III-B): linearise around
 * the iterate, solve the QP with the measured x0, update the iterate
 * (w += dw), send u_0 clamped to [0, u_max], then optionally shift the
 * iterate by one stage (last entries repeated).  x, u are updated in place.
 * status[b] = 0 ok, 4 not positive definite (iterate untouched, u0 = uref).
 * With box != 0 the QP carries the thrust bounds 0 <= u_k + du_k <= u_max
 * (orc_box_qp, at most max_iter subproblems; status 8 if the active sets did
 * not settle, the clamped step is applied); iters[b] receives the number of
 * subproblems solved. */
static void rti_core(const orc_quad* Qd, int nl, const int* w, const double* P, int B, const int* N,
                     const double* dt, const double* Q, const double* R, const double* QN, double* x,
                     double* u, const double* xref, const double* uref, const double* x0m,
                     int shift, double* u0, int* status, int box, int max_iter, int* iters,
                     int second) {
  size_t* xo = (size_t*)malloc(sizeof(size_t) * B);
  size_t* uo = (size_t*)malloc(sizeof(size_t) * B);
  offsets(B, N, xo, uo);
  size_t nn = uo[B - 1] + N[B - 1];
  double* A = (double*)malloc(sizeof(double) * nn * NX * NX);
  double* Bm = (double*)malloc(sizeof(double) * nn * NX * NU);
  double* c = (double*)malloc(sizeof(double) * nn * NX);
  linearize_core(Qd, nl, w, P, B, N, dt, x, u, NULL, NULL, NULL, A, Bm, c, second);
#pragma omp parallel for schedule(dynamic)
  for (int b = 0; b < B; ++b) {
    int Nb = N[b];
    double* xb = x + xo[b] * NX;
    double* ub = u + uo[b] * NU;
    double* dx = (double*)malloc(sizeof(double) * (Nb + 1) * NX);
    double* du = (double*)malloc(sizeof(double) * Nb * NU);
    int st, it = 1;
    if (box) {
      double* lb = (double*)malloc(sizeof(double) * Nb * NU);
      double* hb = (double*)malloc(sizeof(double) * Nb * NU);
      for (int i = 0; i < Nb * NU; ++i) { lb[i] = -ub[i]; hb[i] = Qd->u_max - ub[i]; }
      st = orc_box_qp(NX, NU, Nb, A + uo[b] * NX * NX, Bm + uo[b] * NX * NU, c + uo[b] * NX, xb, ub,
                      xref + xo[b] * NX, uref + uo[b] * NU, Q, R, QN, x0m + b * NX, lb, hb,
                      max_iter, dx, du, &it);
      free(lb); free(hb);
    } else {
      st = orc_riccati(NX, NU, Nb, A + uo[b] * NX * NX, Bm + uo[b] * NX * NU, c + uo[b] * NX, xb,
                       ub, xref + xo[b] * NX, uref + uo[b] * NU, Q, R, QN, x0m + b * NX, dx, du,
                       NULL, NULL);
    }
    status[b] = st;
    if (iters) iters[b] = it;
    if (st == 0 || st == 8) {
      for (int i = 0; i < (Nb + 1) * NX; ++i) xb[i] += dx[i];
      for (int i = 0; i < Nb * NU; ++i) ub[i] += du[i];
      for (int i = 0; i < NU; ++i) {
        double v = ub[i];
        u0[b * NU + i] = v < 0.0 ? 0.0 : (v > Qd->u_max ? Qd->u_max : v);
      }
      if (shift) {
        for (int k = 0; k < Nb; ++k) memcpy(xb + k * NX, xb + (k + 1) * NX, sizeof(double) * NX);
        for (int k = 0; k + 1 < Nb; ++k) memcpy(ub + k * NU, ub + (k + 1) * NU, sizeof(double) * NU);
      }
    } else {
      for (int i = 0; i < NU; ++i) u0[b * NU + i] = uref[uo[b] * NU + i];
    }
    free(dx); free(du);
  }
  free(A); free(Bm); free(c); free(xo); free(uo);
}

void orc_rti_step(const orc_quad* Qd, int nl, const int* w, const double* P, int B, const int* N,
                  const double* dt, const double* Q, const double* R, const double* QN, double* x,
                  double* u, const double* xref, const double* uref, const double* x0m,
                  int shift, double* u0, int* status) {
  rti_core(Qd, nl, w, P, B, N, dt, Q, R, QN, x, u, xref, uref, x0m, shift, u0, status, 0, 0, NULL, 0);
}

/* RTI step with the second-order local model of Eq. 4 */
void orc_rti_step2(const orc_quad* Qd, int nl, const int* w, const double* P, int B, const int* N,
                   const double* dt, const double* Q, const double* R, const double* QN, double* x,
                   double* u, const double* xref, const double* uref, const double* x0m,
                   int shift, double* u0, int* status) {
  rti_core(Qd, nl, w, P, B, N, dt, Q, R, QN, x, u, xref, uref, x0m, shift, u0, status, 0, 0, NULL, 1);
}

void orc_rti_step_box(const orc_quad* Qd, int nl, const int* w, const double* P, int B,
                      const int* N, const double* dt, const double* Q, const double* R,
                      const double* QN, double* x, double* u, const double* xref,
                      const double* uref, const double* x0m, int shift, int max_iter, double* u0,
                      int* status, int* iters) {
  rti_core(Qd, nl, w, P, B, N, dt, Q, R, QN, x, u, xref, uref, x0m, shift, u0, status, 1, max_iter,
           iters, 0);
}

/* Closed loop: each control step runs one RTI step from the plant's state,
 * applies u_0 to the plant for dt (nsub RK4 sub-steps of the true dynamics,
 * then quaternion renormalisation).  References are sampled on each
 * instance's own dt grid: xrt [B][T][13], urt [B][T-1][4] with
 * T >= steps + max N + 1.  The iterate starts at x_k = x0, u_k = hover.
 * traj[steps][B][13] receives the plant state after every step. */
static void closed_loop_core(const orc_quad* Qd, int nl, const int* w, const double* P,
                             int plant_kind, int pnl, const int* pw, const double* PP, int B,
                             const int* N, const double* dt, const double* Q, const double* R,
                             const double* QN, const double* x0, const double* xrt,
                             const double* urt, int T, int steps, double* traj, double* u0_hist,
                             int box, int max_iter, int second) {
  size_t* xo = (size_t*)malloc(sizeof(size_t) * B);
  size_t* uo = (size_t*)malloc(sizeof(size_t) * B);
  offsets(B, N, xo, uo);
  size_t nx_tot = xo[B - 1] + N[B - 1] + 1, nu_tot = uo[B - 1] + N[B - 1];
  double* x = (double*)malloc(sizeof(double) * nx_tot * NX);
  double* u = (double*)malloc(sizeof(double) * nu_tot * NU);
  double* xr = (double*)malloc(sizeof(double) * nx_tot * NX);
  double* ur = (double*)malloc(sizeof(double) * nu_tot * NU);
  double* xp = (double*)malloc(sizeof(double) * B * NX);
  double* u0 = (double*)malloc(sizeof(double) * B * NU);
  int* st = (int*)malloc(sizeof(int) * B);
  double hover = Qd->mass * Qd->g / 4.0;
  for (int b = 0; b < B; ++b) {
    for (int k = 0; k <= N[b]; ++k) memcpy(x + (xo[b] + k) * NX, x0 + b * NX, sizeof(double) * NX);
    for (int k = 0; k < N[b]; ++k)
      for (int i = 0; i < NU; ++i) u[(uo[b] + k) * NU + i] = hover;
    memcpy(xp + b * NX, x0 + b * NX, sizeof(double) * NX);
  }
  for (int t = 0; t < steps; ++t) {
    for (int b = 0; b < B; ++b) {
      for (int k = 0; k <= N[b]; ++k)
        memcpy(xr + (xo[b] + k) * NX, xrt + ((size_t)b * T + t + k) * NX, sizeof(double) * NX);
      for (int k = 0; k < N[b]; ++k)
        memcpy(ur + (uo[b] + k) * NU, urt + ((size_t)b * (T - 1) + t + k) * NU, sizeof(double) * NU);
    }
    rti_core(Qd, nl, w, P, B, N, dt, Q, R, QN, x, u, xr, ur, xp, 1, u0, st, box, max_iter, NULL, second);
#pragma omp parallel for
    for (int b = 0; b < B; ++b) {
      double xn[NX];
      orc_plant_step(Qd, plant_kind, pnl, pw, PP, xp + b * NX, u0 + b * NU, dt[b], 4, xn);
      memcpy(xp + b * NX, xn, sizeof(xn));
    }
    memcpy(traj + (size_t)t * B * NX, xp, sizeof(double) * B * NX);
    if (u0_hist) memcpy(u0_hist + (size_t)t * B * NU, u0, sizeof(double) * B * NU);
  }
  free(xo); free(uo); free(x); free(u); free(xr); free(ur); free(xp); free(u0); free(st);
}

void orc_closed_loop(const orc_quad* Qd, int nl, const int* w, const double* P, int plant_kind,
                     int pnl, const int* pw, const double* PP, int B, const int* N,
                     const double* dt, const double* Q, const double* R, const double* QN,
                     const double* x0, const double* xrt, const double* urt, int T, int steps,
                     double* traj, double* u0_hist) {
  closed_loop_core(Qd, nl, w, P, plant_kind, pnl, pw, PP, B, N, dt, Q, R, QN, x0, xrt, urt, T,
                   steps, traj, u0_hist, 0, 0, 0);
}

/* The closed loop with the second-order local model of Eq. 4 in every RTI
 * step. */
void orc_closed_loop2(const orc_quad* Qd, int nl, const int* w, const double* P, int plant_kind,
                      int pnl, const int* pw, const double* PP, int B, const int* N,
                      const double* dt, const double* Q, const double* R, const double* QN,
                      const double* x0, const double* xrt, const double* urt, int T, int steps,
                      double* traj, double* u0_hist) {
  closed_loop_core(Qd, nl, w, P, plant_kind, pnl, pw, PP, B, N, dt, Q, R, QN, x0, xrt, urt, T,
                   steps, traj, u0_hist, 0, 0, 1);
}

void orc_closed_loop_box(const orc_quad* Qd, int nl, const int* w, const double* P,
                         int plant_kind, int pnl, const int* pw, const double* PP, int B,
                         const int* N, const double* dt, const double* Q, const double* R,
                         const double* QN, const double* x0, const double* xrt,
                         const double* urt, int T, int steps, int max_iter, double* traj,
                         double* u0_hist) {
  closed_loop_core(Qd, nl, w, P, plant_kind, pnl, pw, PP, B, N, dt, Q, R, QN, x0, xrt, urt, T,
                   steps, traj, u0_hist, 1, max_iter, 0);
}

/* ---------------------------------------------------- double integrator --- */
/* Runtime-analysis model (Sec. IV, Eq. 5): x = (p, v), u the commanded
 * acceleration, f_F = (v, u).  The residual network maps z = (p, v, u) to one
 * output added to dv/dt; f_D* is its first-order local model around the
 * node (Eq. 4).  RK4 (u held) with the sensitivity S = d(stage)/d[x; u]
 * (2 x 3) through the four stages; fbar/J may be NULL (nominal model). */
void orc_di_rk4_lin(const double* x, double u, const double* fbar, const double* J, double dt,
                    double* phi, double* A, double* B) {
  double k[4][2], dk[4][6], xs[2], S[6];
  const double cst[4] = {0.0, 0.5, 0.5, 1.0};
  /* D = d f / d[p, v, u]: f_F contributes (v, u), f_D* its Jacobian row */
  double D[6] = {0.0, 1.0, 0.0, 0.0, 0.0, 1.0};
  if (fbar)
    for (int j = 0; j < 3; ++j) D[3 + j] += J[j];
  for (int s = 0; s < 4; ++s) {
    for (int i = 0; i < 2; ++i) xs[i] = x[i] + (s ? cst[s] * dt * k[s - 1][i] : 0.0);
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 3; ++j)
        S[i * 3 + j] = ((i == j) ? 1.0 : 0.0) + (s ? cst[s] * dt * dk[s - 1][i * 3 + j] : 0.0);
    k[s][0] = xs[1];
    k[s][1] = u;
    if (fbar) k[s][1] += fbar[0] + J[0] * (xs[0] - x[0]) + J[1] * (xs[1] - x[1]);
    /* d k_s / d[x; u] = D_x S + D_u [0 0 1] */
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 3; ++j) {
        double sum = (j == 2) ? D[i * 3 + 2] : 0.0;
        for (int l = 0; l < 2; ++l) sum += D[i * 3 + l] * S[l * 3 + j];
        dk[s][i * 3 + j] = sum;
      }
  }
  for (int i = 0; i < 2; ++i) {
    phi[i] = x[i] + dt / 6.0 * (k[0][i] + 2.0 * k[1][i] + 2.0 * k[2][i] + k[3][i]);
    for (int j = 0; j < 3; ++j) {
      double v = ((i == j) ? 1.0 : 0.0) +
                 dt / 6.0 * (dk[0][i * 3 + j] + 2.0 * dk[1][i * 3 + j] + 2.0 * dk[2][i * 3 + j] +
                             dk[3][i * 3 + j]);
      if (j < 2) A[i * 2 + j] = v;
      else B[i] = v;
    }
  }
}

/* Linearise every node of the double integrator (nl = 0: no network):
 * fD [n_nodes], JD [n_nodes][3], A [n_nodes][2][2], Bm [n_nodes][2], c =
 * phi_k - x_{k+1} [n_nodes][2].  Layout as orc_linearize with nx = 2, nu = 1. */
void orc_di_linearize(int nl, const int* w, const double* P, int B, const int* N, const double* dt,
                      const double* x, const double* u, double* fD, double* JD, double* A,
                      double* Bm, double* c) {
  size_t xs = 0, us = 0;
  for (int b = 0; b < B; ++b) {
    for (int k = 0; k < N[b]; ++k) {
      const double* xk = x + (xs + k) * 2;
      const double uk = u[us + k];
      double f = 0.0, J[3] = {0.0, 0.0, 0.0}, phi[2];
      if (nl > 0) {
        const double z[3] = {xk[0], xk[1], uk};
        orc_mlp_fwd_jac(nl, w, P, z, &f, J);
      }
      orc_di_rk4_lin(xk, uk, nl > 0 ? &f : NULL, J, dt[b], phi, A + (us + k) * 4, Bm + (us + k) * 2);
      for (int i = 0; i < 2; ++i) c[(us + k) * 2 + i] = phi[i] - xk[2 + i];
      if (fD) fD[us + k] = f;
      if (JD)
        for (int j = 0; j < 3; ++j) JD[(us + k) * 3 + j] = J[j];
    }
    xs += N[b] + 1;
    us += N[b];
  }
}

/* One RTI step of the double integrator for every instance: linearise
 * around the iterate, solve the QP (orc_riccati, nx = 2, nu = 1) with the
 * measured x0, update the iterate (w += dw), send u_0 (this model has no
 * input bounds), then optionally shift.  status[b] = 0 ok, 4 not positive
 * definite (iterate untouched, u0 = uref). */
void orc_di_rti_step(int nl, const int* w, const double* P, int B, const int* N, const double* dt,
                     const double* Q, const double* R, const double* QN, double* x, double* u,
                     const double* xref, const double* uref, const double* x0m, int shift,
                     double* u0, int* status) {
  size_t nn = 0;
  for (int b = 0; b < B; ++b) nn += N[b];
  double* A = (double*)malloc(sizeof(double) * nn * 4);
  double* Bm = (double*)malloc(sizeof(double) * nn * 2);
  double* c = (double*)malloc(sizeof(double) * nn * 2);
  orc_di_linearize(nl, w, P, B, N, dt, x, u, NULL, NULL, A, Bm, c);
  size_t xs = 0, us = 0;
  for (int b = 0; b < B; ++b) {
    const int Nb = N[b];
    double* xb = x + xs * 2;
    double* ub = u + us;
    double* dx = (double*)malloc(sizeof(double) * (Nb + 1) * 2);
    double* du = (double*)malloc(sizeof(double) * Nb);
    int st = orc_riccati(2, 1, Nb, A + us * 4, Bm + us * 2, c + us * 2, xb, ub, xref + xs * 2,
                         uref + us, Q, R, QN, x0m + b * 2, dx, du, NULL, NULL);
    status[b] = st;
    if (st == 0) {
      for (int i = 0; i < (Nb + 1) * 2; ++i) xb[i] += dx[i];
      for (int i = 0; i < Nb; ++i) ub[i] += du[i];
      u0[b] = ub[0];
      if (shift) {
        for (int k = 0; k < Nb; ++k) memcpy(xb + k * 2, xb + (k + 1) * 2, sizeof(double) * 2);
        for (int k = 0; k + 1 < Nb; ++k) ub[k] = ub[k + 1];
      }
    } else {
      u0[b] = uref[us];
    }
    free(dx); free(du);
    xs += Nb + 1;
    us += Nb;
  }
  free(A); free(Bm); free(c);
}

/* ------------------------------------------------------------ training --- */

/* Mean-squared-error loss over a batch, L = 1/(n * nout) sum |MLP(z) - y|^2,
 * and its gradient with respect to all parameters (packed like P) by
 * backpropagation.  Returns the loss. */
double orc_mse_grad(int nl, const int* w, const double* P, int n, const double* Z,
                    const double* Y, double* G) {
  int hm = mlp_max_width(nl, w), nout = w[nl];
  size_t np = 0;
  for (int l = 0; l < nl; ++l) np += (size_t)w[l + 1] * w[l] + w[l + 1];
  memset(G, 0, sizeof(double) * np);
  double* acts = (double*)malloc(sizeof(double) * hm * (nl + 1));
  double* g = (double*)malloc(sizeof(double) * hm);
  double* g2 = (double*)malloc(sizeof(double) * hm);
  size_t* off = (size_t*)malloc(sizeof(size_t) * (nl + 1));
  off[0] = 0;
  for (int l = 0; l < nl; ++l) off[l + 1] = off[l] + (size_t)w[l + 1] * w[l] + w[l + 1];
  double loss = 0.0, scale = 1.0 / ((double)n * nout);
  for (int s = 0; s < n; ++s) {
    for (int i = 0; i < w[0]; ++i) acts[i] = Z[(size_t)s * w[0] + i];
    for (int l = 0; l < nl; ++l) {
      int fi = w[l], fo = w[l + 1];
      const double* W = P + off[l];
      const double* b = W + (size_t)fo * fi;
      for (int i = 0; i < fo; ++i) {
        double t = b[i];
        for (int k = 0; k < fi; ++k) t += W[(size_t)i * fi + k] * acts[l * hm + k];
        acts[(l + 1) * hm + i] = (l < nl - 1) ? tanh(t) : t;
      }
    }
    for (int i = 0; i < nout; ++i) {
      double e = acts[nl * hm + i] - Y[(size_t)s * nout + i];
      loss += e * e;
      g[i] = 2.0 * e * scale;
    }
    for (int l = nl - 1; l >= 0; --l) {
      int fi = w[l], fo = w[l + 1];
      const double* W = P + off[l];
      double* GW = G + off[l];
      double* Gb = GW + (size_t)fo * fi;
      if (l < nl - 1)
        for (int i = 0; i < fo; ++i) {
          double th = acts[(l + 1) * hm + i];
          g[i] *= 1.0 - th * th;
        }
      for (int i = 0; i < fo; ++i) {
        Gb[i] += g[i];
        for (int k = 0; k < fi; ++k) GW[(size_t)i * fi + k] += g[i] * acts[l * hm + k];
      }
      for (int k = 0; k < fi; ++k) {
        double t = 0.0;
        for (int i = 0; i < fo; ++i) t += W[(size_t)i * fi + k] * g[i];
        g2[k] = t;
      }
      for (int k = 0; k < fi; ++k) g[k] = g2[k];
    }
  }
  free(acts); free(g); free(g2); free(off);
  return loss * scale;
}

/* Adam (Kingma & Ba) with bias correction, step index t >= 1 */
void orc_adam(size_t np, double* P, const double* G, double* m, double* v, int t, double lr,
              double b1, double b2, double eps) {
  double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
  for (size_t i = 0; i < np; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * G[i];
    v[i] = b2 * v[i] + (1.0 - b2) * G[i] * G[i];
    double mh = m[i] / c1, vh = v[i] / c2;
    P[i] -= lr * mh / (sqrt(vh) + eps);
  }
}

/* drag residual targets for a set of samples: Y[n][3] */
void orc_drag_targets(int n, const double* X, double* Y) {
  for (int s = 0; s < n; ++s) orc_drag(X + (size_t)s * NX, Y + (size_t)s * 3);
}
