// Quadrature-point physics of the monolithic ALE fluid-structure step.
//
// Sec. 2 of Margenberg & Richter: ALE fluid, Eq. (ALE) with the stress of
// Eq. (ALE:stress); St. Venant-Kirchhoff solid, Eq. (stress); the shifted
// Crank-Nicolson step of Sec. 2.3 with the forms of Eq. (semiforms).
//
// Conventions: (grad v)_{ij} = d v_i / d x_j, F = I + grad u, J = det F.
// In 2D the adjugate A = J F^{-1} and the cofactor C = J F^{-T} = A^T are
// linear in grad u, which keeps most terms polynomial:
//   J grad v F^{-1} v          = G A v
//   J sigma_f F^{-T}           = (rho nu / J)(G A C + C G^T C) - p C
//   J F^{-1} : grad v^T        = tr(G A)
//   outflow correction          = -(rho nu / J) C G^T C n
// Every flux is written per test slot: for test component c the slot a = 0
// multiplies the test function value, a = 1, 2 its x / y derivative.
//   c = 0, 1  momentum (common test function phi of Eq. (variational))
//   c = 2, 3  displacement rows: kinematic (solid cells, value slot) or
//             harmonic mesh extension (fluid cells, derivative slots)
//   c = 4     divergence row (fluid cells, value slot)
#pragma once

// 2 x 2 matrices of the scalar type R: double for the residual and the FP64
// tangent, float for the tangent of FP32 element matrices.
template <typename R>
struct M2T {
  R a, b, c, d;  // [[a, b], [c, d]]
};
using M2 = M2T<double>;

__host__ __device__ inline M2 m2(double a, double b, double c, double d) { return M2{a, b, c, d}; }
template <typename R>
__host__ __device__ inline M2T<R> operator+(M2T<R> x, M2T<R> y) {
  return M2T<R>{x.a + y.a, x.b + y.b, x.c + y.c, x.d + y.d};
}
template <typename R>
__host__ __device__ inline M2T<R> operator-(M2T<R> x, M2T<R> y) {
  return M2T<R>{x.a - y.a, x.b - y.b, x.c - y.c, x.d - y.d};
}
template <typename R>
__host__ __device__ inline M2T<R> operator*(R s, M2T<R> x) {
  return M2T<R>{s * x.a, s * x.b, s * x.c, s * x.d};
}
template <typename R>
__host__ __device__ inline M2T<R> mul(M2T<R> x, M2T<R> y) {
  return M2T<R>{x.a * y.a + x.b * y.c, x.a * y.b + x.b * y.d, x.c * y.a + x.d * y.c, x.c * y.b + x.d * y.d};
}
template <typename R>
__host__ __device__ inline M2T<R> tp(M2T<R> x) { return M2T<R>{x.a, x.c, x.b, x.d}; }
template <typename R>
__host__ __device__ inline R det(M2T<R> x) { return x.a * x.d - x.b * x.c; }
template <typename R>
__host__ __device__ inline M2T<R> adj(M2T<R> x) { return M2T<R>{x.d, -x.b, -x.c, x.a}; }   // adj(F) = det(F) F^{-1}
template <typename R>
__host__ __device__ inline R trace(M2T<R> x) { return x.a + x.d; }
template <typename R>
__host__ __device__ inline void mv(M2T<R> x, const R* v, R* out) {
  out[0] = x.a * v[0] + x.b * v[1];
  out[1] = x.c * v[0] + x.d * v[1];
}
template <typename R>
__host__ __device__ inline M2T<R> eye2t() { return M2T<R>{R(1), R(0), R(0), R(1)}; }
__host__ __device__ inline M2 eye2() { return eye2t<double>(); }

struct Phys {
  double rho_f, nu_f, rho_s, mu_s, lambda_s;
  double vbar, ramp_t, H, y0;
  double alpha0;
};

// State at one quadrature point: new and old values and gradients.
template <typename R>
struct QpInT {
  R v[2], u[2], p;
  M2T<R> G, Hu;         // grad v, grad u at t_n
  R vo[2], uo[2];
  M2T<R> Go, Huo;       // grad v, grad u at t_{n-1}
};
using QpIn = QpInT<double>;

// Quantities shared by the flux and its linearisation.
template <typename R>
struct QpDerivedT {
  M2T<R> F, A, C, Q;    // t_n: F, adj F, cof F, Q = G A C + C G^T C
  R J;
  M2T<R> Fo, Ao, Co, Qo;
  R Jo;
  M2T<R> Gh, Bh;        // midpoint grad v, F_{n-1/2}^{-1}
  R Jh;                 // (J_{n-1} + J_n) / 2
  R w[2];               // u_n - u_{n-1}
  R M[2];               // Gh Bh w
  // products shared by every direction of the linearisation
  R invJ, invJ2;        // 1 / J, 1 / J^2
  R Bw[2], Av[2];       // Bh w, A v
  M2T<R> GhBh, GA, AC, GtC, CGt;   // Gh Bh, G A, A C, G^T C, C G^T
};
using QpDerived = QpDerivedT<double>;

template <typename R>
__device__ inline void derive(const QpInT<R>& q, QpDerivedT<R>& d) {
  d.F = eye2t<R>() + q.Hu;
  d.J = det(d.F);
  d.A = adj(d.F);
  d.C = tp(d.A);
  d.Q = mul(mul(q.G, d.A), d.C) + mul(mul(d.C, tp(q.G)), d.C);
  d.Fo = eye2t<R>() + q.Huo;
  d.Jo = det(d.Fo);
  d.Ao = adj(d.Fo);
  d.Co = tp(d.Ao);
  d.Qo = mul(mul(q.Go, d.Ao), d.Co) + mul(mul(d.Co, tp(q.Go)), d.Co);
  d.Gh = R(0.5) * (q.G + q.Go);
  M2T<R> Fh = eye2t<R>() + R(0.5) * (q.Hu + q.Huo);
  d.Bh = (R(1.0) / det(Fh)) * adj(Fh);
  d.Jh = R(0.5) * (d.J + d.Jo);
  d.w[0] = q.u[0] - q.uo[0];
  d.w[1] = q.u[1] - q.uo[1];
  mv(d.Bh, d.w, d.Bw);
  mv(d.Gh, d.Bw, d.M);
  d.invJ = R(1.0) / d.J;
  d.invJ2 = d.invJ * d.invJ;
  mv(d.A, q.v, d.Av);
  d.GhBh = mul(d.Gh, d.Bh);
  d.GA = mul(q.G, d.A);
  d.AC = mul(d.A, d.C);
  d.GtC = mul(tp(q.G), d.C);
  d.CGt = mul(d.C, tp(q.G));
}

// First Piola stress of the St. Venant-Kirchhoff solid: F (2 mu E + lambda tr E I).
__device__ inline M2 first_piola(M2 F, double mu, double lam) {
  M2 E = 0.5 * (mul(tp(F), F) - eye2());
  double trE = trace(E);
  M2 S = 2.0 * mu * E + (lam * trE) * eye2();
  return mul(F, S);
}

// Residual flux at a volume quadrature point: out[c * 3 + a].
__device__ inline void qp_flux(const Phys& P, const QpIn& q, const QpDerived& d, bool solid, double k,
                               double theta, double* out) {
  for (int i = 0; i < 15; ++i) out[i] = 0.0;
  const double kt = k * theta, kto = k * (1.0 - theta);
  if (!solid) {
    const double rf = P.rho_f, rn = P.rho_f * P.nu_f;
    double Av[2], GAv[2], Aov[2], GoAov[2];
    mv(d.A, q.v, Av);
    mv(q.G, Av, GAv);
    mv(d.Ao, q.vo, Aov);
    mv(q.Go, Aov, GoAov);
    for (int c = 0; c < 2; ++c) {
      double mass = rf * d.Jh * ((q.v[c] - q.vo[c]) - d.M[c]);
      out[c * 3] = mass + kt * rf * GAv[c] + kto * rf * GoAov[c];
    }
    M2 S = kt * ((rn / d.J) * d.Q - q.p * d.C) + kto * ((rn / d.Jo) * d.Qo - q.p * d.Co);
    out[1] = S.a; out[2] = S.b; out[4] = S.c; out[5] = S.d;
    M2 Hh = kt * q.Hu + kto * q.Huo;            // harmonic extension, Sec. 2.1
    out[7] = Hh.a; out[8] = Hh.b; out[10] = Hh.c; out[11] = Hh.d;
    out[12] = k * trace(mul(q.G, d.A));          // J F^{-1} : grad v^T
  } else {
    M2 Pn = first_piola(d.F, P.mu_s, P.lambda_s), Po = first_piola(d.Fo, P.mu_s, P.lambda_s);
    M2 S = kt * Pn + kto * Po;
    for (int c = 0; c < 2; ++c) {
      out[c * 3] = P.rho_s * (q.v[c] - q.vo[c]);
      out[6 + c * 3] = (q.u[c] - q.uo[c]) - (kt * q.v[c] + kto * q.vo[c]);   // kinematic row
    }
    out[1] = S.a; out[2] = S.b; out[4] = S.c; out[5] = S.d;
  }
}

// Directional derivative of qp_flux in the direction (dv, dG, du, dH, dp) of
// the t_n unknowns: out[c * 3 + a].
template <typename R>
__device__ inline void qp_flux_lin(const Phys& P, const QpInT<R>& q, const QpDerivedT<R>& d, bool solid, R k,
                                   R theta, const R* dv, M2T<R> dG, const R* du, M2T<R> dH, R dp, R* out) {
  for (int i = 0; i < 15; ++i) out[i] = R(0.0);
  const R kt = k * theta, kto = k * (R(1.0) - theta);
  if (!solid) {
    const R rf = R(P.rho_f), rn = R(P.rho_f * P.nu_f);
    const R dJ = trace(mul(d.A, dH));           // d det F = tr(adj(F) dF)
    const M2T<R> dA = adj(dH);                   // adj is linear in 2D
    const M2T<R> dC = tp(dA);
    // ALE mass / domain convection term with midpoint means:
    // d(Gh Bh w) = dGh Bh w + Gh dBh w + Gh Bh dw, dBh = -Bh dFh Bh, dFh = dH / 2
    const R dJh = R(0.5) * dJ;
    R t1[2], t2[2], t3[2], t4[2], dM[2];
    mv(dG, d.Bw, t2);
    mv(dH, d.Bw, t1);
    mv(d.GhBh, t1, t3);
    mv(d.GhBh, du, t4);
    for (int c = 0; c < 2; ++c) dM[c] = R(0.5) * t2[c] - R(0.5) * t3[c] + t4[c];
    // convection G A v
    R dGAv[2], GdAv[2], GAdv[2];
    mv(dG, d.Av, dGAv);
    mv(dA, q.v, t1);
    mv(q.G, t1, GdAv);
    mv(d.GA, dv, GAdv);
    for (int c = 0; c < 2; ++c) {
      out[c * 3] = rf * (dJh * ((q.v[c] - q.vo[c]) - d.M[c]) + d.Jh * (dv[c] - dM[c])) +
                   kt * rf * (dGAv[c] + GdAv[c] + GAdv[c]);
    }
    // stress (rho nu / J) Q - p C, Q = G A C + C G^T C
    M2T<R> dQ = mul(dG, d.AC) + mul(mul(q.G, dA), d.C) + mul(d.GA, dC) + mul(dC, d.GtC) +
                mul(mul(d.C, tp(dG)), d.C) + mul(d.CGt, dC);
    M2T<R> S = kt * ((rn * d.invJ) * dQ - (rn * dJ * d.invJ2) * d.Q - dp * d.C - q.p * dC) - (kto * dp) * d.Co;
    out[1] = S.a; out[2] = S.b; out[4] = S.c; out[5] = S.d;
    M2T<R> Hh = kt * dH;
    out[7] = Hh.a; out[8] = Hh.b; out[10] = Hh.c; out[11] = Hh.d;
    out[12] = k * (trace(mul(dG, d.A)) + trace(mul(q.G, dA)));
  } else {
    const R mu = R(P.mu_s), lam = R(P.lambda_s);
    M2T<R> E = R(0.5) * (mul(tp(d.F), d.F) - eye2t<R>());
    M2T<R> Sig = R(2.0) * mu * E + (lam * trace(E)) * eye2t<R>();
    M2T<R> dE = R(0.5) * (mul(tp(dH), d.F) + mul(tp(d.F), dH));
    M2T<R> dSig = R(2.0) * mu * dE + (lam * trace(dE)) * eye2t<R>();
    M2T<R> S = kt * (mul(dH, Sig) + mul(d.F, dSig));
    for (int c = 0; c < 2; ++c) {
      out[c * 3] = R(P.rho_s) * dv[c];
      out[6 + c * 3] = du[c] - kt * dv[c];
    }
    out[1] = S.a; out[2] = S.b; out[4] = S.c; out[5] = S.d;
  }
}

// Do-nothing correction on the outflow boundary x = x_max (normal n = e_x):
// -k theta (rho nu / J) C G^T C n - k (1 - theta) (rho nu / J_o) C_o G_o^T C_o n,
// value slot of the momentum rows. Only gradients enter.
__device__ inline void edge_flux(const Phys& P, M2 G, M2 Hu, M2 Go, M2 Huo, double k, double theta, double* out) {
  const double rn = P.rho_f * P.nu_f;
  M2 F = eye2() + Hu, Fo = eye2() + Huo;
  M2 C = tp(adj(F)), Co = tp(adj(Fo));
  M2 T = mul(mul(C, tp(G)), C), To = mul(mul(Co, tp(Go)), Co);
  double J = det(F), Jo = det(Fo);
  out[0] = -k * theta * rn / J * T.a - k * (1.0 - theta) * rn / Jo * To.a;
  out[1] = -k * theta * rn / J * T.c - k * (1.0 - theta) * rn / Jo * To.c;
}

template <typename R>
__device__ inline void edge_flux_lin(const Phys& P, M2T<R> G, M2T<R> Hu, M2T<R> dG, M2T<R> dH, R k, R theta,
                                     R* out) {
  const R rn = R(P.rho_f * P.nu_f);
  M2T<R> F = eye2t<R>() + Hu;
  M2T<R> A = adj(F), C = tp(A);
  R J = det(F);
  R dJ = trace(mul(A, dH));
  M2T<R> dC = tp(adj(dH));
  M2T<R> Gt = tp(G);
  M2T<R> T = mul(mul(C, Gt), C);
  M2T<R> dT = mul(mul(dC, Gt), C) + mul(mul(C, tp(dG)), C) + mul(mul(C, Gt), dC);
  M2T<R> Rv = (-k * theta * rn) * ((R(1.0) / J) * dT - (dJ / (J * J)) * T);
  out[0] = Rv.a;
  out[1] = Rv.c;
}

// Directional derivative of qp_flux with respect to the t_{n-1} state
// (dvo, dGo, duo, dHuo); the old pressure does not enter the step. Used by the
// discrete adjoint (the old-state Jacobian dR_n / dU_{n-1}).
__device__ inline void qp_flux_lin_old(const Phys& P, const QpIn& q, const QpDerived& d, bool solid, double k,
                                       double theta, const double* dvo, M2 dGo, const double* duo, M2 dHo,
                                       double* out) {
  for (int i = 0; i < 15; ++i) out[i] = 0.0;
  const double kto = k * (1.0 - theta);
  if (!solid) {
    const double rf = P.rho_f, rn = P.rho_f * P.nu_f;
    const double dJo = trace(mul(d.Ao, dHo));
    const M2 dAo = adj(dHo);
    const M2 dCo = tp(dAo);
    // ALE mass term: J_{n-1/2}, grad v_{n-1/2}, F_{n-1/2} and u_n - u_{n-1} depend on the old state
    const double dJh = 0.5 * dJo;
    const M2 dGh = 0.5 * dGo;
    const M2 dBh = -0.5 * mul(mul(d.Bh, dHo), d.Bh);
    double t1[2], t2[2], t3[2], t4[2], dM[2], mdw[2] = {-duo[0], -duo[1]};
    mv(d.Bh, d.w, t1);
    mv(dGh, t1, t2);
    mv(dBh, d.w, t1);
    mv(d.Gh, t1, t3);
    mv(d.Bh, mdw, t1);
    mv(d.Gh, t1, t4);
    for (int c = 0; c < 2; ++c) dM[c] = t2[c] + t3[c] + t4[c];
    // old convection G_o A_o v_o
    double Aov[2], dGAv[2], GdAv[2], GAdv[2];
    mv(d.Ao, q.vo, Aov);
    mv(dGo, Aov, dGAv);
    mv(dAo, q.vo, t1);
    mv(q.Go, t1, GdAv);
    mv(d.Ao, dvo, t1);
    mv(q.Go, t1, GAdv);
    for (int c = 0; c < 2; ++c)
      out[c * 3] = rf * (dJh * ((q.v[c] - q.vo[c]) - d.M[c]) + d.Jh * (-dvo[c] - dM[c])) +
                   kto * rf * (dGAv[c] + GdAv[c] + GAdv[c]);
    // old stress (rho nu / J_o) Q_o - p_n C_o
    M2 Gt = tp(q.Go), dGt = tp(dGo);
    M2 dQ = mul(mul(dGo, d.Ao), d.Co) + mul(mul(q.Go, dAo), d.Co) + mul(mul(q.Go, d.Ao), dCo) +
            mul(mul(dCo, Gt), d.Co) + mul(mul(d.Co, dGt), d.Co) + mul(mul(d.Co, Gt), dCo);
    M2 S = kto * ((rn / d.Jo) * dQ - (rn * dJo / (d.Jo * d.Jo)) * d.Qo - q.p * dCo);
    out[1] = S.a; out[2] = S.b; out[4] = S.c; out[5] = S.d;
    M2 Hh = kto * dHo;
    out[7] = Hh.a; out[8] = Hh.b; out[10] = Hh.c; out[11] = Hh.d;
  } else {
    const double mu = P.mu_s, lam = P.lambda_s;
    M2 E = 0.5 * (mul(tp(d.Fo), d.Fo) - eye2());
    M2 Sig = 2.0 * mu * E + (lam * trace(E)) * eye2();
    M2 dE = 0.5 * (mul(tp(dHo), d.Fo) + mul(tp(d.Fo), dHo));
    M2 dSig = 2.0 * mu * dE + (lam * trace(dE)) * eye2();
    M2 S = kto * (mul(dHo, Sig) + mul(d.Fo, dSig));
    for (int c = 0; c < 2; ++c) {
      out[c * 3] = -P.rho_s * dvo[c];
      out[6 + c * 3] = -duo[c] - kto * dvo[c];
    }
    out[1] = S.a; out[2] = S.b; out[4] = S.c; out[5] = S.d;
  }
}

// Old-state part of the outflow correction, -k (1 - theta)(rho nu / J_o) C_o G_o^T C_o n.
__device__ inline void edge_flux_lin_old(const Phys& P, M2 Go, M2 Huo, M2 dGo, M2 dHo, double k, double theta,
                                         double* out) {
  edge_flux_lin(P, Go, Huo, dGo, dHo, k, 1.0 - theta, out);
}

// Derivatives of the solid first Piola stress F Sigma with respect to the Lame
// parameters: dP/dmu = F 2E, dP/dlambda = F tr(E) I.
__device__ inline M2 dpiola_dmu(M2 F) {
  M2 E = 0.5 * (mul(tp(F), F) - eye2());
  return mul(F, 2.0 * E);
}
__device__ inline M2 dpiola_dlambda(M2 F) {
  M2 E = 0.5 * (mul(tp(F), F) - eye2());
  return trace(E) * F;
}
