// Element residuals of the monolithic ALE FSI system on P1 tetrahedra.
//
// One routine per element kind, templated on the scalar S of the unknowns
// (T = double / float for the residual, Dual<T> for one Jacobian column) and the
// base type T of constant data (reference coordinates, previous time levels).
//
//   fluid tets : ALE Navier-Stokes momentum and continuity on the current tet
//                x = X + d (Sec. 2.1, Eq. 3; backward Euler, Eq. 9), stabilised
//                by SUPG / PSPG / LSIC (P1-P1 pair, Sec. 2.2), plus the harmonic
//                mesh-motion operator on the reference tet (Eq. 1).
//   wall tets  : St. Venant-Kirchhoff wall momentum in total Lagrangian form,
//                F = I + grad d, E = (F^T F - I)/2, S = lambda tr E I + 2 mu E,
//                Pi = F S (Sec. 2.1, Eq. 2), consistent P1 mass, BE in time.
//
// Stabilisation constants (the paper defers them to its references):
//   h = (6 sqrt2 |K_0|)^(1/3) on the reference tet,
//   D = sqrt((2 rho/dt)^2 + (2 rho |a_c|/h)^2 + (4 mu/h^2)^2), a_c = (u - w) at the
//   centroid, tau_M = rho/D (SUPG), tau_M/rho = 1/D (PSPG), tau_C rho = h^2 D/12.
// The 4-point degree-2 rule integrates every term exactly for P1 fields.
#pragma once
#include "dual.cuh"

namespace fsi {

struct MatConst {
  double rho_f, mu_f, rho_s, eta_s, lam_s, mu_s, dt;
};

// barycentric weights of the degree-2 4-point rule: alpha at its own vertex,
// beta at the three others; each point carries weight 1/4
#define FSI_QA 0.5854101966249685
#define FSI_QB 0.1381966011250105

// shape-function gradients g[4][3] and volume of the tet with vertices x[4][3]
template <class S>
__device__ __forceinline__ void tet_gradients(const S x[4][3], S g[4][3], S& vol) {
  S e[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) e[k][i] = x[k + 1][i] - x[0][i];
  // rows of the inverse edge matrix: cross products of the other two edges / det
  S c[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int p = (k + 1) % 3, q = (k + 2) % 3;
    c[k][0] = e[p][1] * e[q][2] - e[p][2] * e[q][1];
    c[k][1] = e[p][2] * e[q][0] - e[p][0] * e[q][2];
    c[k][2] = e[p][0] * e[q][1] - e[p][1] * e[q][0];
  }
  S det = e[0][0] * c[0][0] + e[0][1] * c[0][1] + e[0][2] * c[0][2];
  S inv = S(1) / det;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    g[1][i] = c[0][i] * inv;
    g[2][i] = c[1][i] * inv;
    g[3][i] = c[2][i] * inv;
    g[0][i] = -(g[1][i] + g[2][i] + g[3][i]);
  }
  vol = det / S(6);
}

// Fluid tet. Inputs: reference vertices X, unknowns u, p, d at the vertices, the
// previous level u1, d1. Outputs (overwritten): momentum Rm[a][i], continuity
// Rc[a], mesh motion Rh[a][i].
template <class S, class T>
__device__ __forceinline__ void fluid_element(const T X[4][3], const S u[4][3], const S p[4],
                                              const S d[4][3], const T u1[4][3], const T d1[4][3],
                                              const MatConst& m, S Rm[4][3], S Rc[4], S Rh[4][3]) {
  const T rho = T(m.rho_f), mu = T(m.mu_f), dt = T(m.dt);
  const T idt = T(1) / dt;
  // current geometry (ALE map) and reference geometry
  S x[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) x[a][i] = X[a][i] + d[a][i];
  S g[4][3], vol;
  tet_gradients<S>(x, g, vol);
  T g0[4][3], vol0;
  tet_gradients<T>(X, g0, vol0);

  // velocity gradient G_ij = du_i/dx_j, divergence, pressure gradient
  S G[3][3], gp[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) G[i][j] = u[0][i] * g[0][j] + u[1][i] * g[1][j] + u[2][i] * g[2][j] + u[3][i] * g[3][j];
    gp[i] = p[0] * g[0][i] + p[1] * g[1][i] + p[2] * g[2][i] + p[3] * g[3][i];
  }
  S divu = G[0][0] + G[1][1] + G[2][2];

  // ALE advection velocity a = u - w, w = (d - d_old)/dt
  S ae[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) ae[a][i] = u[a][i] - (d[a][i] - d1[a][i]) * idt;
  S ac[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) ac[i] = (ae[0][i] + ae[1][i] + ae[2][i] + ae[3][i]) * T(0.25);

  // stabilisation parameters (constant per tet)
  const T h = cbrt(T(6) * sqrt(T(2)) * vol0);
  const T ih2 = T(1) / (h * h);
  const T c_t = T(2) * rho * idt;
  const T c_v = T(4) * mu * ih2;
  S aa = ac[0] * ac[0] + ac[1] * ac[1] + ac[2] * ac[2];
  S D = dsqrt(c_t * c_t + (T(4) * rho * rho * ih2) * aa + c_v * c_v);
  S tau_m = rho / D;
  S tau_p = S(1) / D;
  S tau_c = (h * h / T(12)) * D;

#pragma unroll
  for (int a = 0; a < 4; ++a) {
    Rc[a] = S(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) Rm[a][i] = S(0);
  }

  const S wv = vol * T(0.25);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    T N[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) N[a] = (a == q) ? T(FSI_QA) : T(FSI_QB);
    S uq[3], aq[3];
    T u1q[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      uq[i] = N[0] * u[0][i] + N[1] * u[1][i] + N[2] * u[2][i] + N[3] * u[3][i];
      aq[i] = N[0] * ae[0][i] + N[1] * ae[1][i] + N[2] * ae[2][i] + N[3] * ae[3][i];
      u1q[i] = N[0] * u1[0][i] + N[1] * u1[1][i] + N[2] * u1[2][i] + N[3] * u1[3][i];
    }
    S inert[3], rM[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      S conv = G[i][0] * aq[0] + G[i][1] * aq[1] + G[i][2] * aq[2];
      inert[i] = rho * (uq[i] - u1q[i]) * idt + rho * conv;
      rM[i] = inert[i] + gp[i];
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      S adv = aq[0] * g[a][0] + aq[1] * g[a][1] + aq[2] * g[a][2];
      S supg = tau_m * adv;
#pragma unroll
      for (int i = 0; i < 3; ++i) Rm[a][i] += wv * (N[a] * inert[i] + supg * rM[i]);
      S gr = g[a][0] * rM[0] + g[a][1] * rM[1] + g[a][2] * rM[2];
      Rc[a] += wv * (N[a] * divu + tau_p * gr);
    }
  }

  // pressure, viscous and grad-div terms: constant integrands for P1
  S pc = (p[0] + p[1] + p[2] + p[3]) * T(0.25);
  S lsic = tau_c * divu;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      S visc = (G[i][0] + G[0][i]) * g[a][0] + (G[i][1] + G[1][i]) * g[a][1] + (G[i][2] + G[2][i]) * g[a][2];
      Rm[a][i] += vol * ((lsic - pc) * g[a][i] + mu * visc);
    }
  }

  // harmonic mesh motion on the reference tet: |K0| sum_b (g0_a . g0_b) d_b
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    T kab[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) kab[b] = vol0 * (g0[a][0] * g0[b][0] + g0[a][1] * g0[b][1] + g0[a][2] * g0[b][2]);
#pragma unroll
    for (int i = 0; i < 3; ++i) Rh[a][i] = kab[0] * d[0][i] + kab[1] * d[1][i] + kab[2] * d[2][i] + kab[3] * d[3][i];
  }
}

// Wall tet: momentum residual Rw[a][i] for displacement d (unknown), d1 = d_{n-1},
// d2 = d_{n-2}.
template <class S, class T>
__device__ __forceinline__ void wall_element(const T X[4][3], const S d[4][3], const T d1[4][3],
                                             const T d2[4][3], const MatConst& m, S Rw[4][3]) {
  const T idt = T(1) / T(m.dt);
  T g0[4][3], vol0;
  tet_gradients<T>(X, g0, vol0);
  // deformation gradient F = I + sum_a d_a (x) g0_a
  S F[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      F[i][j] = d[0][i] * g0[0][j] + d[1][i] * g0[1][j] + d[2][i] * g0[2][j] + d[3][i] * g0[3][j] + (i == j ? T(1) : T(0));
  // Green-Lagrange strain, second Piola-Kirchhoff stress, first Piola-Kirchhoff
  S E[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      E[i][j] = T(0.5) * (F[0][i] * F[0][j] + F[1][i] * F[1][j] + F[2][i] * F[2][j] - (i == j ? T(1) : T(0)));
  S trE = E[0][0] + E[1][1] + E[2][2];
  S Sg[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Sg[i][j] = T(2) * T(m.mu_s) * E[i][j] + (i == j ? T(m.lam_s) * trE : S(0));
  S P[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) P[i][j] = F[i][0] * Sg[0][j] + F[i][1] * Sg[1][j] + F[i][2] * Sg[2][j];
  // inertia (consistent mass (1 + delta_ab)|K0|/20) and damping
  S acc[4][3];
#pragma unroll
  for (int b = 0; b < 4; ++b)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      S vs = (d[b][i] - d1[b][i]) * idt;
      T vs1 = (d1[b][i] - d2[b][i]) * idt;
      acc[b][i] = T(m.rho_s) * (vs - vs1) * idt + T(m.eta_s) * vs;
    }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      S sum = acc[0][i] + acc[1][i] + acc[2][i] + acc[3][i] + acc[a][i];
      Rw[a][i] = vol0 * ((T(1) / T(20)) * sum + P[i][0] * g0[a][0] + P[i][1] * g0[a][1] + P[i][2] * g0[a][2]);
    }
}

}  // namespace fsi
