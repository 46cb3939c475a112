// Element physics of the monolithic ALE fluid-structure step in 3D: hexahedral
// Q2 cells (27 nodes, 3 x 3 x 3 Gauss points), 7 unknowns per node
// (v_x, v_y, v_z, u_x, u_y, u_z, p).
//
// Sec. 2 of Margenberg & Richter: ALE fluid, Eq. (ALE) with the stress of
// Eq. (ALE:stress); St. Venant-Kirchhoff solid, Eq. (stress); the shifted
// Crank-Nicolson step of Sec. 2.3 with the forms of Eq. (semiforms). The 2D
// kernels use the same readings; in 3D the adjugate A = J F^{-1} and the
// cofactor C = A^T are quadratic in grad u, and the terms keep the 2D shape:
//   J grad v F^{-1} v          = G A v
//   J sigma_f F^{-T}           = (rho nu / J)(G A C + C G^T C) - p C
//   J F^{-1} : grad v^T        = tr(G A)
//   outflow correction          = -(rho nu / J) C G^T C n,   n = e_x
// Fluxes are written per test slot: out[c * 4 + a], a = 0 the test function
// value, a = 1, 2, 3 its x / y / z derivative; c = 0-2 momentum, 3-5
// displacement rows (kinematic on solid cells, harmonic extension on fluid
// cells), 6 the divergence row.
//
// Everything here is __host__ __device__: the CUDA kernels and host-side checks
// compile the same code.
#pragma once

#include <cmath>

#include "fsi_cta.h"

#ifdef __CUDACC__
#define FSI3_HD __host__ __device__
#else
#define FSI3_HD
#endif

namespace fsi3 {

struct M3 {
  double m[3][3];
};

FSI3_HD inline M3 eye3() {
  M3 r{};
  r.m[0][0] = r.m[1][1] = r.m[2][2] = 1.0;
  return r;
}
FSI3_HD inline M3 add(const M3& x, const M3& y) {
  M3 r;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) r.m[i][j] = x.m[i][j] + y.m[i][j];
  return r;
}
FSI3_HD inline M3 scale(double s, const M3& x) {
  M3 r;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) r.m[i][j] = s * x.m[i][j];
  return r;
}
FSI3_HD inline M3 mul(const M3& x, const M3& y) {
  M3 r;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) r.m[i][j] = x.m[i][0] * y.m[0][j] + x.m[i][1] * y.m[1][j] + x.m[i][2] * y.m[2][j];
  return r;
}
FSI3_HD inline M3 tp(const M3& x) {
  M3 r;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) r.m[i][j] = x.m[j][i];
  return r;
}
FSI3_HD inline double det(const M3& x) {
  const double (*a)[3] = x.m;
  return a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) - a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
         a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
}
// adj(x): x adj(x) = det(x) I
FSI3_HD inline M3 adj(const M3& x) {
  const double (*a)[3] = x.m;
  M3 r;
  r.m[0][0] = a[1][1] * a[2][2] - a[1][2] * a[2][1];
  r.m[0][1] = a[0][2] * a[2][1] - a[0][1] * a[2][2];
  r.m[0][2] = a[0][1] * a[1][2] - a[0][2] * a[1][1];
  r.m[1][0] = a[1][2] * a[2][0] - a[1][0] * a[2][2];
  r.m[1][1] = a[0][0] * a[2][2] - a[0][2] * a[2][0];
  r.m[1][2] = a[0][2] * a[1][0] - a[0][0] * a[1][2];
  r.m[2][0] = a[1][0] * a[2][1] - a[1][1] * a[2][0];
  r.m[2][1] = a[0][1] * a[2][0] - a[0][0] * a[2][1];
  r.m[2][2] = a[0][0] * a[1][1] - a[0][1] * a[1][0];
  return r;
}
FSI3_HD inline double trace(const M3& x) { return x.m[0][0] + x.m[1][1] + x.m[2][2]; }
FSI3_HD inline void mv(const M3& x, const double* v, double* out) {
  for (int i = 0; i < 3; ++i) out[i] = x.m[i][0] * v[0] + x.m[i][1] * v[1] + x.m[i][2] * v[2];
}

struct Phys3 {
  double rho_f, nu_f, rho_s, mu_s, lambda_s;
};

// New and old values and gradients at one quadrature point.
struct Qp3 {
  double v[3], u[3], p;
  M3 G, Hu;      // grad v, grad u at t_n
  double vo[3], uo[3];
  M3 Go, Huo;    // at t_{n-1}
};

// Residual fluxes at a volume quadrature point, out[28] (see the header).
FSI3_HD inline void qp_flux3(const Phys3& P, const Qp3& q, bool solid, double k, double theta, double* out) {
  for (int i = 0; i < 28; ++i) out[i] = 0.0;
  const double kt = k * theta, kto = k * (1.0 - theta);
  const M3 I = eye3();
  const M3 F = add(I, q.Hu), Fo = add(I, q.Huo);
  if (!solid) {
    const double rf = P.rho_f, rn = P.rho_f * P.nu_f;
    const double J = det(F), Jo = det(Fo);
    const M3 A = adj(F), Ao = adj(Fo), C = tp(A), Co = tp(Ao);
    // ALE mass term with midpoint means: Jh ((v - vo) - Gh Fh^{-1} (u - uo))
    M3 Gh = scale(0.5, add(q.G, q.Go));
    M3 Fh = add(I, scale(0.5, add(q.Hu, q.Huo)));
    const M3 Bh = scale(1.0 / det(Fh), adj(Fh));
    const double Jh = 0.5 * (J + Jo);
    double w[3], t[3], M[3], Av[3], GAv[3], Aov[3], GoAov[3];
    for (int c = 0; c < 3; ++c) w[c] = q.u[c] - q.uo[c];
    mv(Bh, w, t);
    mv(Gh, t, M);
    mv(A, q.v, Av);
    mv(q.G, Av, GAv);
    mv(Ao, q.vo, Aov);
    mv(q.Go, Aov, GoAov);
    for (int c = 0; c < 3; ++c)
      out[c * 4] = rf * Jh * ((q.v[c] - q.vo[c]) - M[c]) + kt * rf * GAv[c] + kto * rf * GoAov[c];
    // stress: (rho nu / J)(G A C + C G^T C) - p C, old geometry with the new pressure
    const M3 Q = add(mul(mul(q.G, A), C), mul(mul(C, tp(q.G)), C));
    const M3 Qo = add(mul(mul(q.Go, Ao), Co), mul(mul(Co, tp(q.Go)), Co));
    for (int c = 0; c < 3; ++c)
      for (int j = 0; j < 3; ++j)
        out[c * 4 + 1 + j] = kt * ((rn / J) * Q.m[c][j] - q.p * C.m[c][j]) +
                             kto * ((rn / Jo) * Qo.m[c][j] - q.p * Co.m[c][j]);
    // harmonic mesh extension
    for (int c = 0; c < 3; ++c)
      for (int j = 0; j < 3; ++j) out[(3 + c) * 4 + 1 + j] = kt * q.Hu.m[c][j] + kto * q.Huo.m[c][j];
    out[6 * 4] = k * trace(mul(q.G, A));
  } else {
    auto piola = [&](const M3& Fx) {
      M3 E = scale(0.5, add(mul(tp(Fx), Fx), scale(-1.0, I)));
      const double trE = trace(E);
      M3 S = add(scale(2.0 * P.mu_s, E), scale(P.lambda_s * trE, I));
      return mul(Fx, S);
    };
    const M3 S = add(scale(kt, piola(F)), scale(kto, piola(Fo)));
    for (int c = 0; c < 3; ++c) {
      out[c * 4] = P.rho_s * (q.v[c] - q.vo[c]);
      out[(3 + c) * 4] = (q.u[c] - q.uo[c]) - (kt * q.v[c] + kto * q.vo[c]);
      for (int j = 0; j < 3; ++j) out[c * 4 + 1 + j] = S.m[c][j];
    }
  }
}

// Do-nothing correction on the outflow face x = x_max (value slot of the
// momentum rows): -k theta (rho nu / J) C G^T C e_x - k (1 - theta) (...)_{n-1}.
FSI3_HD inline void face_flux3(const Phys3& P, const M3& G, const M3& Hu, const M3& Go, const M3& Huo, double k,
                               double theta, double* out) {
  const double rn = P.rho_f * P.nu_f;
  const M3 I = eye3();
  const M3 F = add(I, Hu), Fo = add(I, Huo);
  const M3 C = tp(adj(F)), Co = tp(adj(Fo));
  const M3 T = mul(mul(C, tp(G)), C), To = mul(mul(Co, tp(Go)), Co);
  const double J = det(F), Jo = det(Fo);
  for (int c = 0; c < 3; ++c) out[c] = -k * theta * rn / J * T.m[c][0] - k * (1.0 - theta) * rn / Jo * To.m[c][0];
}

// Directional derivative of qp_flux3 in the direction (dv, dG, du, dH, dp) of
// the t_n unknowns, out[28]. In 3D the adjugate is quadratic in grad u:
// d adj(F)[dH] = (tr(A dH) A - A dH A) / J (from adj F = J F^{-1}).
// The parts of the linearised flux at one point that do not depend on the
// direction (state, old state and material only): computed once per point and
// shared by its 28 directions.
struct Qp3Lin {
  M3 F, A, C, Co, Gh, Bh, Gt, Q, Sig, AC;
  double J, Jh, w[3], Bw[3], M[3], Av[3];
};

FSI3_HD inline void qp_lin_prepare3(const Phys3& P, const Qp3& q, bool solid, Qp3Lin& L) {
  const M3 I = eye3();
  L.F = add(I, q.Hu);
  if (!solid) {
    const M3 Fo = add(I, q.Huo);
    L.J = det(L.F);
    const double Jo = det(Fo);
    L.A = adj(L.F);
    L.C = tp(L.A);
    L.Co = tp(adj(Fo));
    L.Gh = scale(0.5, add(q.G, q.Go));
    const M3 Fh = add(I, scale(0.5, add(q.Hu, q.Huo)));
    L.Bh = scale(1.0 / det(Fh), adj(Fh));
    L.Jh = 0.5 * (L.J + Jo);
    for (int c = 0; c < 3; ++c) L.w[c] = q.u[c] - q.uo[c];
    mv(L.Bh, L.w, L.Bw);
    mv(L.Gh, L.Bw, L.M);
    mv(L.A, q.v, L.Av);
    L.Gt = tp(q.G);
    L.Q = add(mul(mul(q.G, L.A), L.C), mul(mul(L.C, L.Gt), L.C));
    L.AC = mul(L.A, L.C);
  } else {
    const double mu = P.mu_s, lam = P.lambda_s;
    const M3 E = scale(0.5, add(mul(tp(L.F), L.F), scale(-1.0, I)));
    L.Sig = add(scale(2.0 * mu, E), scale(lam * trace(E), I));
  }
}

// The linearised flux at one point in one direction, from the prepared parts.
FSI3_HD inline void qp_flux3_lin_prepared(const Phys3& P, const Qp3& q, const Qp3Lin& L, bool solid, double k,
                                          double theta, const double* dv, const M3& dG, const double* du,
                                          const M3& dH, double dp, double* out) {
  for (int i = 0; i < 28; ++i) out[i] = 0.0;
  const double kt = k * theta, kto = k * (1.0 - theta);
  if (!solid) {
    const double rf = P.rho_f, rn = P.rho_f * P.nu_f;
    const M3& A = L.A;
    const M3& C = L.C;
    const double J = L.J;
    const double dJ = trace(mul(A, dH));
    const M3 dA = scale(1.0 / J, add(scale(dJ, A), scale(-1.0, mul(mul(A, dH), A))));
    const M3 dC = tp(dA);
    // mass term: Jh ((v - vo) - Gh Bh w), Bh = Fh^{-1}, dBh = -Bh (dH / 2) Bh
    const double dJh = 0.5 * dJ;
    const M3 dBh = scale(-0.5, mul(mul(L.Bh, dH), L.Bh));
    double t1[3], t2[3], t3[3], t4[3], dM[3];
    mv(dG, L.Bw, t1);               // dGh Bh w = (dG / 2) Bh w
    mv(dBh, L.w, t2);
    mv(L.Gh, t2, t3);               // Gh dBh w
    mv(L.Bh, du, t2);
    mv(L.Gh, t2, t4);               // Gh Bh dw
    for (int c = 0; c < 3; ++c) dM[c] = 0.5 * t1[c] + t3[c] + t4[c];
    // convection G A v
    double dGAv[3], dAv[3], GdAv[3], Adv[3], GAdv[3];
    mv(dG, L.Av, dGAv);
    mv(dA, q.v, dAv);
    mv(q.G, dAv, GdAv);
    mv(A, dv, Adv);
    mv(q.G, Adv, GAdv);
    for (int c = 0; c < 3; ++c)
      out[c * 4] = rf * (dJh * ((q.v[c] - q.vo[c]) - L.M[c]) + L.Jh * (dv[c] - dM[c])) +
                   kt * rf * (dGAv[c] + GdAv[c] + GAdv[c]);
    // stress (rho nu / J) Q - p C with Q = G A C + C G^T C; the old term depends on p only
    const M3 dGt = tp(dG);
    const M3& Gt = L.Gt;
    M3 dQ = add(add(mul(mul(dG, A), C), mul(mul(q.G, dA), C)), mul(mul(q.G, A), dC));
    dQ = add(dQ, add(add(mul(mul(dC, Gt), C), mul(mul(C, dGt), C)), mul(mul(C, Gt), dC)));
    for (int c = 0; c < 3; ++c)
      for (int j = 0; j < 3; ++j)
        out[c * 4 + 1 + j] = kt * ((rn / J) * dQ.m[c][j] - (rn * dJ / (J * J)) * L.Q.m[c][j] - dp * C.m[c][j] -
                                   q.p * dC.m[c][j]) -
                             kto * dp * L.Co.m[c][j];
    for (int c = 0; c < 3; ++c)
      for (int j = 0; j < 3; ++j) out[(3 + c) * 4 + 1 + j] = kt * dH.m[c][j];
    out[6 * 4] = k * (trace(mul(dG, A)) + trace(mul(q.G, dA)));
  } else {
    const double mu = P.mu_s, lam = P.lambda_s;
    const M3& F = L.F;
    const M3 dE = scale(0.5, add(mul(tp(dH), F), mul(tp(F), dH)));
    const M3 dSig = add(scale(2.0 * mu, dE), scale(lam * trace(dE), eye3()));
    const M3 S = scale(kt, add(mul(dH, L.Sig), mul(F, dSig)));
    for (int c = 0; c < 3; ++c) {
      out[c * 4] = P.rho_s * dv[c];
      out[(3 + c) * 4] = du[c] - kt * dv[c];
      for (int j = 0; j < 3; ++j) out[c * 4 + 1 + j] = S.m[c][j];
    }
  }
}

// The linearised flux in one unit direction: trial field cj (v, u components,
// then p), slot b (0: the value, 1 + d: the derivative in direction d). Only
// the nine displacement-gradient directions need dense 3 x 3 products; the
// others reduce to rank-one updates or vanish. Equal to
// qp_flux3_lin_prepared in the same direction up to rounding.
FSI3_HD inline void qp_flux3_lin_unit(const Phys3& P, const Qp3& q, const Qp3Lin& L, bool solid, double k,
                                      double theta, int cj, int b, double* out) {
  for (int i = 0; i < 28; ++i) out[i] = 0.0;
  const double kt = k * theta, kto = k * (1.0 - theta);
  if (solid) {
    if (cj < 3) {
      if (b == 0) {
        out[cj * 4] = P.rho_s;
        out[(3 + cj) * 4] = -kt;
      }
    } else if (cj < 6) {
      const int c = cj - 3;
      if (b == 0) {
        out[(3 + c) * 4] = 1.0;
      } else {
        const int j = b - 1;   // dH = e_c e_j^T
        const double mu = P.mu_s, lam = P.lambda_s;
        const M3& F = L.F;
        M3 dSig;
        const double trE = F.m[c][j];
        for (int r = 0; r < 3; ++r)
          for (int t = 0; t < 3; ++t) {
            const double dE = 0.5 * ((r == j ? F.m[c][t] : 0.0) + (t == j ? F.m[c][r] : 0.0));
            dSig.m[r][t] = 2.0 * mu * dE + (r == t ? lam * trE : 0.0);
          }
        const M3 FdS = mul(F, dSig);
        for (int r = 0; r < 3; ++r)
          for (int t = 0; t < 3; ++t) out[r * 4 + 1 + t] = kt * ((r == c ? L.Sig.m[j][t] : 0.0) + FdS.m[r][t]);
      }
    }
    return;
  }
  const double rf = P.rho_f, rn = P.rho_f * P.nu_f;
  const M3& A = L.A;
  const M3& C = L.C;
  const double J = L.J;
  if (cj < 3) {
    const int c = cj;
    if (b == 0) {   // dv = e_c: mass and convection G A e_c
      for (int r = 0; r < 3; ++r) {
        double gac = 0.0;
        for (int t = 0; t < 3; ++t) gac += q.G.m[r][t] * A.m[t][c];
        out[r * 4] = rf * (L.Jh * (r == c ? 1.0 : 0.0)) + kt * rf * gac;
      }
      return;
    }
    const int j = b - 1;   // dG = e_c e_j^T
    out[c * 4] = rf * (L.Jh * (-0.5 * L.Bw[j])) + kt * rf * L.Av[j];
    for (int r = 0; r < 3; ++r)
      for (int t = 0; t < 3; ++t) {
        const double dQ = (r == c ? L.AC.m[j][t] : 0.0) + C.m[r][j] * C.m[c][t];
        out[r * 4 + 1 + t] = kt * ((rn / J) * dQ);
      }
    out[6 * 4] = k * A.m[j][c];
    return;
  }
  if (cj < 6) {
    const int c = cj - 3;
    if (b == 0) {   // du = e_c: the mesh-velocity part of the mass term, Gh Bh e_c
      double t2[3] = {L.Bh.m[0][c], L.Bh.m[1][c], L.Bh.m[2][c]}, t4[3];
      mv(L.Gh, t2, t4);
      for (int r = 0; r < 3; ++r) out[r * 4] = rf * (L.Jh * (0.0 - t4[r]));
      return;
    }
    const int j = b - 1;   // dH = e_c e_j^T
    const double dJ = A.m[j][c];
    M3 dA, dBh;
    for (int r = 0; r < 3; ++r)
      for (int t = 0; t < 3; ++t) {
        dA.m[r][t] = (1.0 / J) * (dJ * A.m[r][t] - A.m[r][c] * A.m[j][t]);
        dBh.m[r][t] = -0.5 * (L.Bh.m[r][c] * L.Bh.m[j][t]);
      }
    const M3 dC = tp(dA);
    double t2[3], dM[3], dAv[3], GdAv[3];
    mv(dBh, L.w, t2);
    mv(L.Gh, t2, dM);
    mv(dA, q.v, dAv);
    mv(q.G, dAv, GdAv);
    const double dJh = 0.5 * dJ;
    for (int r = 0; r < 3; ++r)
      out[r * 4] = rf * (dJh * ((q.v[r] - q.vo[r]) - L.M[r]) + L.Jh * (0.0 - dM[r])) + kt * rf * GdAv[r];
    const M3& Gt = L.Gt;
    const M3 dQ = add(add(mul(mul(q.G, dA), C), mul(mul(q.G, A), dC)),
                      add(mul(mul(dC, Gt), C), mul(mul(C, Gt), dC)));
    for (int r = 0; r < 3; ++r)
      for (int t = 0; t < 3; ++t)
        out[r * 4 + 1 + t] = kt * ((rn / J) * dQ.m[r][t] - (rn * dJ / (J * J)) * L.Q.m[r][t] - q.p * dC.m[r][t]);
    out[(3 + c) * 4 + 1 + j] = kt;
    out[6 * 4] = k * trace(mul(q.G, dA));
    return;
  }
  if (b == 0)   // dp = 1
    for (int r = 0; r < 3; ++r)
      for (int t = 0; t < 3; ++t) out[r * 4 + 1 + t] = kt * (-C.m[r][t]) - kto * L.Co.m[r][t];
}

FSI3_HD inline void qp_flux3_lin(const Phys3& P, const Qp3& q, bool solid, double k, double theta, const double* dv,
                                 const M3& dG, const double* du, const M3& dH, double dp, double* out) {
  Qp3Lin L;
  qp_lin_prepare3(P, q, solid, L);
  qp_flux3_lin_prepared(P, q, L, solid, k, theta, dv, dG, du, dH, dp, out);
}

// Directional derivative of face_flux3 in the t_n gradients (dG, dH), out[3].
FSI3_HD inline void face_flux3_lin(const Phys3& P, const M3& G, const M3& Hu, const M3& dG, const M3& dH, double k,
                                   double theta, double* out) {
  const double rn = P.rho_f * P.nu_f;
  const M3 F = add(eye3(), Hu);
  const double J = det(F);
  const M3 A = adj(F), C = tp(A);
  const double dJ = trace(mul(A, dH));
  const M3 dC = tp(scale(1.0 / J, add(scale(dJ, A), scale(-1.0, mul(mul(A, dH), A)))));
  const M3 Gt = tp(G);
  const M3 T = mul(mul(C, Gt), C);
  const M3 dT = add(add(mul(mul(dC, Gt), C), mul(mul(C, tp(dG)), C)), mul(mul(C, Gt), dC));
  for (int c = 0; c < 3; ++c) out[c] = -k * theta * rn * (dT.m[c][0] / J - dJ / (J * J) * T.m[c][0]);
}

// Reference tables of the Q2 hexahedron on the unit cube. Node l = a + 3 b + 9 c
// and quadrature point q likewise (x fastest); the outflow face s_x = 1 has the
// 9 Gauss points of its (y, z) plane. lps[a][l][m] = integral over the unit cube
// of d_a kappa(phi_l) d_a kappa(phi_m), kappa = I - (Q1 vertex interpolation).
struct Tables3 {
  double phi[27][27], dphi[3][27][27];     // [q][l], [dir][q][l]
  double wq[27];
  double phi_f[9][27], dphi_f[3][9][27];   // outflow face
  double wf[9];
  double lps[3][27][27];
  double g1v[3][3], g1d[3][3];             // 1D: lag2(i, gp[s]), dlag2(i, gp[s]) [i][s]
};

inline double lag2(int a, double s) {
  return a == 0 ? (1 - s) * (1 - 2 * s) : (a == 1 ? 4 * s * (1 - s) : s * (2 * s - 1));
}
inline double dlag2(int a, double s) { return a == 0 ? 4 * s - 3 : (a == 1 ? 4 - 8 * s : 4 * s - 1); }

inline void build_tables3(Tables3& T) {
  const double gp[3] = {0.5 - std::sqrt(0.15), 0.5, 0.5 + std::sqrt(0.15)};
  const double gw[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  auto idx = [](int l, int* a) { a[0] = l % 3; a[1] = (l / 3) % 3; a[2] = l / 9; };
  for (int i = 0; i < 3; ++i)
    for (int q = 0; q < 3; ++q) {
      T.g1v[i][q] = lag2(i, gp[q]);
      T.g1d[i][q] = dlag2(i, gp[q]);
    }
  for (int q = 0; q < 27; ++q) {
    int qi[3];
    idx(q, qi);
    T.wq[q] = gw[qi[0]] * gw[qi[1]] * gw[qi[2]];
    for (int l = 0; l < 27; ++l) {
      int li[3];
      idx(l, li);
      double v[3], dv[3];
      for (int a = 0; a < 3; ++a) {
        v[a] = lag2(li[a], gp[qi[a]]);
        dv[a] = dlag2(li[a], gp[qi[a]]);
      }
      T.phi[q][l] = v[0] * v[1] * v[2];
      T.dphi[0][q][l] = dv[0] * v[1] * v[2];
      T.dphi[1][q][l] = v[0] * dv[1] * v[2];
      T.dphi[2][q][l] = v[0] * v[1] * dv[2];
    }
  }
  for (int f = 0; f < 9; ++f) {
    const int fy = f % 3, fz = f / 3;
    T.wf[f] = gw[fy] * gw[fz];
    for (int l = 0; l < 27; ++l) {
      int li[3];
      idx(l, li);
      const double vx = lag2(li[0], 1.0), dx = dlag2(li[0], 1.0);
      const double vy = lag2(li[1], gp[fy]), dy = dlag2(li[1], gp[fy]);
      const double vz = lag2(li[2], gp[fz]), dz = dlag2(li[2], gp[fz]);
      T.phi_f[f][l] = vx * vy * vz;
      T.dphi_f[0][f][l] = dx * vy * vz;
      T.dphi_f[1][f][l] = vx * dy * vz;
      T.dphi_f[2][f][l] = vx * vy * dz;
    }
  }
  // kappa(phi_l) gradients: subtract the Q1 vertex function for vertex nodes
  double gk[3][27][27];   // [dir][q][l]
  for (int q = 0; q < 27; ++q) {
    int qi[3];
    idx(q, qi);
    for (int l = 0; l < 27; ++l) {
      int li[3];
      idx(l, li);
      const bool vertex = li[0] != 1 && li[1] != 1 && li[2] != 1;
      for (int d = 0; d < 3; ++d) {
        double g1 = 0.0;
        if (vertex) {
          g1 = 1.0;
          for (int a = 0; a < 3; ++a) {
            const double s = gp[qi[a]];
            const int vtx = li[a] / 2;   // 0 or 1
            const double val = vtx ? s : 1 - s, der = vtx ? 1.0 : -1.0;
            g1 *= (a == d) ? der : val;
          }
        }
        gk[d][q][l] = T.dphi[d][q][l] - g1;
      }
    }
  }
  for (int d = 0; d < 3; ++d)
    for (int l = 0; l < 27; ++l)
      for (int m = 0; m < 27; ++m) {
        double s = 0.0;
        for (int q = 0; q < 27; ++q) s += T.wq[q] * gk[d][q][l] * gk[d][q][m];
        T.lps[d][l][m] = s;
      }
}

// Residual contributions of one cell, Re[l * 7 + c] (before the row selection
// of the assembly): Ue, Uo the cell's nodal values [27][7] at t_n and t_{n-1},
// h the cell's edge lengths, alpha its stabilisation weight.
FSI3_HD inline void cell_residual3(const Phys3& P, const Tables3& T, const double* Ue, const double* Uo,
                                   const double* h, bool solid, bool outflow, double k, double theta, double alpha,
                                   double* Re) {
  for (int i = 0; i < 27 * 7; ++i) Re[i] = 0.0;
  const double vol = h[0] * h[1] * h[2];
  for (int q = 0; q < 27; ++q) {
    Qp3 x{};
    for (int l = 0; l < 27; ++l) {
      const double ph = T.phi[q][l];
      const double g[3] = {T.dphi[0][q][l] / h[0], T.dphi[1][q][l] / h[1], T.dphi[2][q][l] / h[2]};
      for (int c = 0; c < 3; ++c) {
        x.v[c] += ph * Ue[l * 7 + c];
        x.u[c] += ph * Ue[l * 7 + 3 + c];
        x.vo[c] += ph * Uo[l * 7 + c];
        x.uo[c] += ph * Uo[l * 7 + 3 + c];
        for (int j = 0; j < 3; ++j) {
          x.G.m[c][j] += g[j] * Ue[l * 7 + c];
          x.Hu.m[c][j] += g[j] * Ue[l * 7 + 3 + c];
          x.Go.m[c][j] += g[j] * Uo[l * 7 + c];
          x.Huo.m[c][j] += g[j] * Uo[l * 7 + 3 + c];
        }
      }
      x.p += ph * Ue[l * 7 + 6];
    }
    double f[28];
    qp_flux3(P, x, solid, k, theta, f);
    const double W = T.wq[q] * vol;
    for (int l = 0; l < 27; ++l) {
      const double ph = T.phi[q][l];
      const double g[3] = {T.dphi[0][q][l] / h[0], T.dphi[1][q][l] / h[1], T.dphi[2][q][l] / h[2]};
      for (int c = 0; c < 7; ++c)
        Re[l * 7 + c] += W * (ph * f[c * 4] + g[0] * f[c * 4 + 1] + g[1] * f[c * 4 + 2] + g[2] * f[c * 4 + 3]);
    }
  }
  if (!solid) {   // local projection stabilisation of the divergence rows
    const double s[3] = {vol / (h[0] * h[0]), vol / (h[1] * h[1]), vol / (h[2] * h[2])};
    for (int l = 0; l < 27; ++l) {
      double acc = 0.0;
      for (int m = 0; m < 27; ++m)
        acc += (s[0] * T.lps[0][l][m] + s[1] * T.lps[1][l][m] + s[2] * T.lps[2][l][m]) * Ue[m * 7 + 6];
      Re[l * 7 + 6] += k * alpha * acc;
    }
  }
  if (outflow && !solid) {
    for (int f = 0; f < 9; ++f) {
      M3 G{}, Hu{}, Go{}, Huo{};
      for (int l = 0; l < 27; ++l) {
        const double g[3] = {T.dphi_f[0][f][l] / h[0], T.dphi_f[1][f][l] / h[1], T.dphi_f[2][f][l] / h[2]};
        for (int c = 0; c < 3; ++c)
          for (int j = 0; j < 3; ++j) {
            G.m[c][j] += g[j] * Ue[l * 7 + c];
            Hu.m[c][j] += g[j] * Ue[l * 7 + 3 + c];
            Go.m[c][j] += g[j] * Uo[l * 7 + c];
            Huo.m[c][j] += g[j] * Uo[l * 7 + 3 + c];
          }
      }
      double fo[3];
      face_flux3(P, G, Hu, Go, Huo, k, theta, fo);
      const double W = T.wf[f] * h[1] * h[2];
      for (int l = 0; l < 27; ++l)
        for (int c = 0; c < 3; ++c) Re[l * 7 + c] += W * T.phi_f[f][l] * fo[c];
    }
  }
}

// States, gradients and old values at volume quadrature point q of a cell.
FSI3_HD inline Qp3 qp_state3(const Tables3& T, const double* Ue, const double* Uo, const double* h, int q) {
  Qp3 x{};
  for (int l = 0; l < 27; ++l) {
    const double ph = T.phi[q][l];
    const double g[3] = {T.dphi[0][q][l] / h[0], T.dphi[1][q][l] / h[1], T.dphi[2][q][l] / h[2]};
    for (int c = 0; c < 3; ++c) {
      x.v[c] += ph * Ue[l * 7 + c];
      x.u[c] += ph * Ue[l * 7 + 3 + c];
      x.vo[c] += ph * Uo[l * 7 + c];
      x.uo[c] += ph * Uo[l * 7 + 3 + c];
      for (int jj = 0; jj < 3; ++jj) {
        x.G.m[c][jj] += g[jj] * Ue[l * 7 + c];
        x.Hu.m[c][jj] += g[jj] * Ue[l * 7 + 3 + c];
        x.Go.m[c][jj] += g[jj] * Uo[l * 7 + c];
        x.Huo.m[c][jj] += g[jj] * Uo[l * 7 + 3 + c];
      }
    }
    x.p += ph * Ue[l * 7 + 6];
  }
  return x;
}

// Element matrix of one cell, Ke[(l * 7 + ci) * 189 + m * 7 + cj] = dRe[l, ci] / dUe[m, cj]
// (before the row selection of the assembly), by the two-stage contraction
// K += sum_q W B_l^T D_q B_m with the 28 x 28 tangent D_q of qp_flux3_lin.
FSI3_HD inline void cell_jacobian3(const Phys3& P, const Tables3& T, const double* Ue, const double* Uo,
                                   const double* h, bool solid, bool outflow, double k, double theta, double alpha,
                                   double* Ke) {
  for (int i = 0; i < 189 * 189; ++i) Ke[i] = 0.0;
  const double vol = h[0] * h[1] * h[2];
  for (int q = 0; q < 27; ++q) {
    const Qp3 x = qp_state3(T, Ue, Uo, h, q);
    double D[28][28];   // [test slot ci * 4 + a][trial direction cj * 4 + b]
    for (int dir = 0; dir < 28; ++dir) {
      const int cj = dir / 4, b = dir % 4;
      double dv[3] = {0, 0, 0}, du[3] = {0, 0, 0}, dp = 0.0;
      M3 dG{}, dH{};
      if (cj < 3) {
        if (b == 0) dv[cj] = 1.0;
        else dG.m[cj][b - 1] = 1.0;
      } else if (cj < 6) {
        if (b == 0) du[cj - 3] = 1.0;
        else dH.m[cj - 3][b - 1] = 1.0;
      } else if (b == 0) {
        dp = 1.0;
      }
      double o[28];
      qp_flux3_lin(P, x, solid, k, theta, dv, dG, du, dH, dp, o);
      for (int r = 0; r < 28; ++r) D[r][dir] = o[r];
    }
    const double W = T.wq[q] * vol;
    double B[4][27];
    for (int l = 0; l < 27; ++l) {
      B[0][l] = T.phi[q][l];
      for (int a = 0; a < 3; ++a) B[1 + a][l] = T.dphi[a][q][l] / h[a];
    }
    for (int ci = 0; ci < 7; ++ci)
      for (int cj = 0; cj < 7; ++cj) {
        double E[4][27];   // E[a][m] = sum_b D[ci a][cj b] B_b(m)
        for (int a = 0; a < 4; ++a)
          for (int m = 0; m < 27; ++m) {
            double e = 0.0;
            for (int b = 0; b < 4; ++b) e += D[ci * 4 + a][cj * 4 + b] * B[b][m];
            E[a][m] = W * e;
          }
        for (int l = 0; l < 27; ++l)
          for (int m = 0; m < 27; ++m) {
            double acc = 0.0;
            for (int a = 0; a < 4; ++a) acc += B[a][l] * E[a][m];
            Ke[(l * 7 + ci) * 189 + m * 7 + cj] += acc;
          }
      }
  }
  if (!solid) {
    const double s3[3] = {vol / (h[0] * h[0]), vol / (h[1] * h[1]), vol / (h[2] * h[2])};
    for (int l = 0; l < 27; ++l)
      for (int m = 0; m < 27; ++m)
        Ke[(l * 7 + 6) * 189 + m * 7 + 6] +=
            k * alpha * (s3[0] * T.lps[0][l][m] + s3[1] * T.lps[1][l][m] + s3[2] * T.lps[2][l][m]);
  }
  if (outflow && !solid) {
    for (int f = 0; f < 9; ++f) {
      M3 G{}, Hu{};
      double gf[3][27];
      for (int l = 0; l < 27; ++l) {
        for (int a = 0; a < 3; ++a) gf[a][l] = T.dphi_f[a][f][l] / h[a];
        for (int c = 0; c < 3; ++c)
          for (int jj = 0; jj < 3; ++jj) {
            G.m[c][jj] += gf[jj][l] * Ue[l * 7 + c];
            Hu.m[c][jj] += gf[jj][l] * Ue[l * 7 + 3 + c];
          }
      }
      const double W = T.wf[f] * h[1] * h[2];
      for (int cj = 0; cj < 6; ++cj)
        for (int b = 0; b < 3; ++b) {
          M3 dG{}, dH{};
          if (cj < 3) dG.m[cj][b] = 1.0;
          else dH.m[cj - 3][b] = 1.0;
          double o[3];
          face_flux3_lin(P, G, Hu, dG, dH, k, theta, o);
          for (int l = 0; l < 27; ++l)
            for (int m = 0; m < 27; ++m)
              for (int c = 0; c < 3; ++c) Ke[(l * 7 + c) * 189 + m * 7 + cj] += W * T.phi_f[f][l] * o[c] * gf[b][m];
        }
    }
  }
}

// ---------------------------------------------------------------------------
// The cell residual computed by a cooperative thread group (fsi_cta.h): the
// arithmetic of cell_residual3 in the same order (bit for bit), with the 27
// point fluxes and the 9 outflow-face fluxes computed in parallel and each of
// the 189 entries summed over the points by one thread. Shared scratch
// CR3_TOTAL doubles; the caller stores Ue at CR3_UE and Uo at CR3_UE + 189 and
// synchronises before the call.
// ---------------------------------------------------------------------------
constexpr int CR3_X = 0;                            // Qp3[27]
constexpr int CR3_F = CR3_X + 27 * (int)(sizeof(Qp3) / sizeof(double));   // [27][28] point fluxes
constexpr int CR3_FO = CR3_F + 27 * 28;             // [9][3] face fluxes
constexpr int CR3_UE = CR3_FO + 27;                 // Ue[189], Uo[189]
constexpr int CR3_TOTAL = CR3_UE + 378;

template <class Cta>
FSI3_HD inline void cell_residual3_cta(const Cta& cta, const Phys3& P, const Tables3& T, const double* h, bool solid,
                                       bool outflow, double k, double theta, double alpha, double* sh, double* Re) {
  const double* Ue = sh + CR3_UE;
  const double* Uo = Ue + 189;
  Qp3* X = reinterpret_cast<Qp3*>(sh + CR3_X);
  double* F = sh + CR3_F;
  double* FO = sh + CR3_FO;
  const double vol = h[0] * h[1] * h[2];
  const bool face = outflow && !solid;
  for (int q = cta.tid; q < 27; q += cta.nt) {
    X[q] = qp_state3(T, Ue, Uo, h, q);
    qp_flux3(P, X[q], solid, k, theta, F + q * 28);
  }
  if (face)
    for (int f = cta.tid; f < 9; f += cta.nt) {
      M3 G{}, Hu{}, Go{}, Huo{};
      for (int l = 0; l < 27; ++l) {
        const double g[3] = {T.dphi_f[0][f][l] / h[0], T.dphi_f[1][f][l] / h[1], T.dphi_f[2][f][l] / h[2]};
        for (int c = 0; c < 3; ++c)
          for (int j = 0; j < 3; ++j) {
            G.m[c][j] += g[j] * Ue[l * 7 + c];
            Hu.m[c][j] += g[j] * Ue[l * 7 + 3 + c];
            Go.m[c][j] += g[j] * Uo[l * 7 + c];
            Huo.m[c][j] += g[j] * Uo[l * 7 + 3 + c];
          }
      }
      face_flux3(P, G, Hu, Go, Huo, k, theta, FO + f * 3);
    }
  cta.sync();
  const double s3[3] = {vol / (h[0] * h[0]), vol / (h[1] * h[1]), vol / (h[2] * h[2])};
  for (int e = cta.tid; e < 189; e += cta.nt) {
    const int l = e / 7, c = e % 7;
    double r = 0.0;
    for (int q = 0; q < 27; ++q) {
      const double* f = F + q * 28;
      const double W = T.wq[q] * vol;
      const double ph = T.phi[q][l];
      const double g[3] = {T.dphi[0][q][l] / h[0], T.dphi[1][q][l] / h[1], T.dphi[2][q][l] / h[2]};
      r += W * (ph * f[c * 4] + g[0] * f[c * 4 + 1] + g[1] * f[c * 4 + 2] + g[2] * f[c * 4 + 3]);
    }
    if (!solid && c == 6) {
      double acc = 0.0;
      for (int m = 0; m < 27; ++m)
        acc += (s3[0] * T.lps[0][l][m] + s3[1] * T.lps[1][l][m] + s3[2] * T.lps[2][l][m]) * Ue[m * 7 + 6];
      r += k * alpha * acc;
    }
    if (face && c < 3)
      for (int f = 0; f < 9; ++f) r += T.wf[f] * h[1] * h[2] * T.phi_f[f][l] * FO[f * 3 + c];
    Re[e] = r;
  }
}

// ---------------------------------------------------------------------------
// The element matrix computed by a cooperative thread group (fsi_cta.h), with
// the work spread over the group and each entry of Ke written once. The
// tangent columns of one trial field cj (27 points x 28 test slots x 4
// directions) are computed together. For each test field ci, a (ci, cj) block
// whose tangents vanish at every point is written as zeros (unless the
// pressure stabilisation or the outflow face adds to it). Otherwise
// E[q][a][m] = W_q sum_b D_q[ci a][cj b] B_b(m, q), as in cell_jacobian3, and
// Ke[l ci][m cj] = sum_a sum_q B_a(l, q) E[q][a][m] by sum factorisation: the
// Q2 basis and the 3 x 3 x 3 Gauss rule are tensor products, so B_a(l, q) =
// F1(l1, q1) F2(l2, q2) F3(l3, q3) with F the 1D values, or derivatives / h in
// the direction of a, and the sum over q runs as three 1D contractions (q3,
// then q2, then q1): 3 x 2916 instead of 729 x 108 multiply-adds per block.
// The result equals cell_jacobian3 up to rounding (another summation order).
// Shared scratch (doubles, CJ3_TOTAL); the caller stores Ue at CJ3_UE and Uo
// at CJ3_UE + 189 and synchronises before the call.
// ---------------------------------------------------------------------------
constexpr int CJ3_XSZ = (int)(sizeof(Qp3) / sizeof(double));
constexpr int CJ3_X = 0;                        // Qp3[27]
constexpr int CJ3_B = CJ3_X + 27 * CJ3_XSZ;     // [27 q][4 a][27 l]
constexpr int CJ3_W = CJ3_B + 27 * 4 * 27;      // [27] W_q
constexpr int CJ3_D = CJ3_W + 27;               // [27 q][28 slots][4 b]: columns of the current trial field
constexpr int CJ3_E = CJ3_D + 27 * 28 * 4;      // [27 q][4 a][27 m]
constexpr int CJ3_FG = CJ3_E + 27 * 4 * 27;     // [9 face points][G, Hu]
constexpr int CJ3_FO = CJ3_FG + 9 * 18;         // [9 face points][3 c][3 b] face tangents of the current field
constexpr int CJ3_FLAG = CJ3_FO + 81;           // [7] nonzero flags of the (ci, cj) blocks
constexpr int CJ3_UE = CJ3_FLAG + 8;            // Ue[189], Uo[189]
constexpr int CJ3_T1 = CJ3_UE + 378;            // [4 a][27 m][9 (q1, q2)][3 l3]
constexpr int CJ3_T2 = CJ3_T1 + 2916;           // [4 a][27 m][3 q1][9 (l2, l3)]
constexpr int CJ3_F = CJ3_T2 + 2916;            // [3 d][2: value, derivative / h_d][3 i][3 s]
constexpr int CJ3_LSZ = (int)(sizeof(Qp3Lin) / sizeof(double));
constexpr int CJ3_XL = CJ3_F + 54;              // Qp3Lin[27]: the direction-independent tangent parts
constexpr int CJ3_TOTAL = CJ3_XL + 27 * CJ3_LSZ;
static_assert(sizeof(Qp3) % sizeof(double) == 0, "Qp3 holds doubles only");
static_assert(sizeof(Qp3Lin) % sizeof(double) == 0, "Qp3Lin holds doubles only");

FSI3_HD inline bool cj3_nonzero(double x) {
#ifdef __CUDA_ARCH__
  return (__double_as_longlong(x) << 1) != 0;   // bit test: keeps the FP64 pipe free
#else
  return x != 0.0 || x != x;
#endif
}

template <class Cta>
FSI3_HD inline void cell_jacobian3_cta(const Cta& cta, const Phys3& P, const Tables3& T, const double* h, bool solid,
                                       bool outflow, double k, double theta, double alpha, double* sh, double* Ke) {
  const double* Ue = sh + CJ3_UE;
  const double* Uo = Ue + 189;
  Qp3* X = reinterpret_cast<Qp3*>(sh + CJ3_X);
  double* B = sh + CJ3_B;
  double* Wq = sh + CJ3_W;
  double* Dc = sh + CJ3_D;
  double* E = sh + CJ3_E;
  double* FG = sh + CJ3_FG;
  double* FO = sh + CJ3_FO;
  double* flag = sh + CJ3_FLAG;
  const double vol = h[0] * h[1] * h[2];
  const bool face = outflow && !solid;
  Qp3Lin* XL = reinterpret_cast<Qp3Lin*>(sh + CJ3_XL);
  for (int q = cta.tid; q < 27; q += cta.nt) {
    X[q] = qp_state3(T, Ue, Uo, h, q);
    qp_lin_prepare3(P, X[q], solid, XL[q]);
    Wq[q] = T.wq[q] * vol;
  }
  for (int e = cta.tid; e < 27 * 4 * 27; e += cta.nt) {
    const int q = e / 108, a = (e / 27) % 4, l = e % 27;
    B[e] = a == 0 ? T.phi[q][l] : T.dphi[a - 1][q][l] / h[a - 1];
  }
  if (face)
    for (int f = cta.tid; f < 9; f += cta.nt) {
      M3 G{}, Hu{};
      for (int l = 0; l < 27; ++l) {
        double gf[3];
        for (int a = 0; a < 3; ++a) gf[a] = T.dphi_f[a][f][l] / h[a];
        for (int c = 0; c < 3; ++c)
          for (int jj = 0; jj < 3; ++jj) {
            G.m[c][jj] += gf[jj] * Ue[l * 7 + c];
            Hu.m[c][jj] += gf[jj] * Ue[l * 7 + 3 + c];
          }
      }
      for (int i = 0; i < 9; ++i) {
        FG[f * 18 + i] = G.m[i / 3][i % 3];
        FG[f * 18 + 9 + i] = Hu.m[i / 3][i % 3];
      }
    }
  double* T1 = sh + CJ3_T1;
  double* T2 = sh + CJ3_T2;
  double* F = sh + CJ3_F;
  for (int e = cta.tid; e < 54; e += cta.nt) {
    const int d = e / 18, der = (e / 9) % 2, i = (e / 3) % 3, q = e % 3;
    F[e] = der ? T.g1d[i][q] / h[d] : T.g1v[i][q];
  }
  // F_d(a)(i, s): the 1D factor of B_a in direction d (the derivative where a = d + 1)
  auto Fa = [&](int d, int a, int i, int q) { return F[((d * 2 + (a == d + 1 ? 1 : 0)) * 3 + i) * 3 + q]; };
  const double s3[3] = {vol / (h[0] * h[0]), vol / (h[1] * h[1]), vol / (h[2] * h[2])};
  cta.sync();   // X, XL, Wq, B, FG and F are read below by other threads than their writers
  for (int cj = 0; cj < 7; ++cj) {
    for (int e = cta.tid; e < 27 * 4; e += cta.nt) {
      const int q = e / 4, b = e % 4;
      double o[28];
      qp_flux3_lin_unit(P, X[q], XL[q], solid, k, theta, cj, b, o);
      for (int r = 0; r < 28; ++r) Dc[(q * 28 + r) * 4 + b] = o[r];
    }
    if (face && cj < 6)
      for (int e = cta.tid; e < 27; e += cta.nt) {
        const int f = e / 3, b = e % 3;
        M3 G, Hu, dG{}, dH{};
        for (int i = 0; i < 9; ++i) {
          G.m[i / 3][i % 3] = FG[f * 18 + i];
          Hu.m[i / 3][i % 3] = FG[f * 18 + 9 + i];
        }
        if (cj < 3) dG.m[cj][b] = 1.0;
        else dH.m[cj - 3][b] = 1.0;
        double o[3];
        face_flux3_lin(P, G, Hu, dG, dH, k, theta, o);
        for (int c = 0; c < 3; ++c) FO[(f * 3 + c) * 3 + b] = o[c];
      }
    cta.sync();
    // flag[ci]: whether any tangent entry of test field ci (rows 4 ci .. 4 ci + 3) is nonzero;
    // one warp per field on the device (needs at least 224 threads), one thread per field on the host
#ifdef __CUDA_ARCH__
    if (cta.tid < 7 * 32) {
      const int f = cta.tid / 32, lane = cta.tid % 32;
      bool nz = false;
      for (int e = lane; e < 27 * 16; e += 32) nz |= cj3_nonzero(Dc[((e / 16) * 28 + 4 * f) * 4 + e % 16]);
      nz = __any_sync(0xffffffffu, nz);
      if (lane == 0) flag[f] = nz ? 1.0 : 0.0;
    }
#else
    for (int f = cta.tid; f < 7; f += cta.nt) {
      bool nz = false;
      for (int e = 0; e < 27 * 16; ++e) nz |= cj3_nonzero(Dc[((e / 16) * 28 + 4 * f) * 4 + e % 16]);
      flag[f] = nz ? 1.0 : 0.0;
    }
#endif
    cta.sync();
    for (int ci = 0; ci < 7; ++ci) {
      const bool lps = !solid && ci == 6 && cj == 6, fc = face && ci < 3 && cj < 6;
      if (flag[ci] == 0.0 && !lps && !fc) {
        for (int e = cta.tid; e < 729; e += cta.nt)
          Ke[((e / 27) * 7 + ci) * 189 + (e % 27) * 7 + cj] = 0.0;
        continue;
      }
      for (int e = cta.tid; e < 27 * 4 * 27; e += cta.nt) {
        const int q = e / 108, a = (e / 27) % 4, m = e % 27;
        double ev = 0.0;
        for (int b = 0; b < 4; ++b) ev += Dc[(q * 28 + ci * 4 + a) * 4 + b] * B[(q * 4 + b) * 27 + m];
        E[e] = Wq[q] * ev;
      }
      cta.sync();
      // contract q3: T1[a][m][q1 + 3 q2][l3]
      for (int e = cta.tid; e < 2916; e += cta.nt) {
        const int a = e / 729, m = (e / 27) % 27, q12 = (e / 3) % 9, l3 = e % 3;
        double acc = 0.0;
        for (int q3 = 0; q3 < 3; ++q3) acc += Fa(2, a, l3, q3) * E[((q12 + 9 * q3) * 4 + a) * 27 + m];
        T1[e] = acc;
      }
      cta.sync();
      // contract q2: T2[a][m][q1][l2 + 3 l3]
      for (int e = cta.tid; e < 2916; e += cta.nt) {
        const int a = e / 729, m = (e / 27) % 27, q1 = (e / 9) % 3, l23 = e % 9, l2 = l23 % 3, l3 = l23 / 3;
        double acc = 0.0;
        for (int q2 = 0; q2 < 3; ++q2) acc += Fa(1, a, l2, q2) * T1[((a * 27 + m) * 9 + q1 + 3 * q2) * 3 + l3];
        T2[e] = acc;
      }
      cta.sync();
      // contract q1 and sum over a
      for (int e = cta.tid; e < 729; e += cta.nt) {
        const int l = e / 27, m = e % 27, l1 = l % 3, l23 = l / 3;
        double kv = 0.0;
        for (int a = 0; a < 4; ++a)
          for (int q1 = 0; q1 < 3; ++q1) kv += Fa(0, a, l1, q1) * T2[((a * 27 + m) * 3 + q1) * 9 + l23];
        if (lps) kv += k * alpha * (s3[0] * T.lps[0][l][m] + s3[1] * T.lps[1][l][m] + s3[2] * T.lps[2][l][m]);
        if (fc)
          for (int f = 0; f < 9; ++f) {
            const double W = T.wf[f] * h[1] * h[2];
            for (int b = 0; b < 3; ++b) kv += W * T.phi_f[f][l] * FO[(f * 3 + ci) * 3 + b] * (T.dphi_f[b][f][m] / h[b]);
          }
        Ke[(l * 7 + ci) * 189 + m * 7 + cj] = kv;
      }
      cta.sync();
    }
    cta.sync();
  }
}

// Stabilisation weight of a cell from its old state (the same reading as in
// 2D): alpha = alpha0 h^2 / (rho_f nu_f + rho_f |vbar| h), vbar the Gauss mean
// of v_{n-1} over the cell, h the cell diameter.
FSI3_HD inline double stab_weight3(const Tables3& T, const double* Uo, const double* h, double alpha0, double rho_f,
                                   double nu_f) {
  double vb[3] = {0, 0, 0}, ws = 0.0;
  for (int q = 0; q < 27; ++q) {
    ws += T.wq[q];
    for (int l = 0; l < 27; ++l)
      for (int c = 0; c < 3; ++c) vb[c] += T.wq[q] * T.phi[q][l] * Uo[l * 7 + c];
  }
  const double sp = sqrt(vb[0] * vb[0] + vb[1] * vb[1] + vb[2] * vb[2]) / ws;
  const double hd = sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
  return alpha0 * hd * hd / (rho_f * nu_f + rho_f * sp * hd);
}

}  // namespace fsi3
