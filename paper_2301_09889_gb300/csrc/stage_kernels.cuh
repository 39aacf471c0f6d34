// The two wall-normal halves of one Runge-Kutta stage, each fused over a tile
// of `ppc` Fourier modes that lives in shared memory:
//
//   stage_pre  : (v, omega_y, U, W) coefficients -> coefficients of
//                u, v, w, omega_x, omega_y, omega_z -> their values at the
//                Gauss-Lobatto nodes (input of the nonlinear plane kernel);
//   stage_post : nodal values of H = u x omega -> Chebyshev coefficients ->
//                right-hand sides -> Chebyshev-tau solves -> new state.
//
// Every global array is read and written once per stage with loads and
// stores that are contiguous over the modes of the tile; the sequential
// recurrences then run on shared memory.  RN is the precision of the nodal
// values exchanged with the plane kernel (double: all-FP64 path).
//
// Symmetry classes and components.  All wall-normal operators are real and
// map even Chebyshev coefficients to even or odd ones in a fixed pattern, so a
// mode splits into two classes (c = 0: even v, odd omega_y; c = 1: odd v,
// even omega_y) and two real components (r = 0, 1) that never interact.  The
// factors i kx, i kz only swap components: component r of (i s X) is
// sgn_r s X_{1-r} with sgn_0 = -1, sgn_1 = +1.  One thread owns one
// (mode, class, component[, equation]) and keeps one parity of its arrays in
// registers (parity index i, n = 2i + sig), bounded at compile time by MH.
//
// Chebyshev conventions: f(y) = sum_n a_n T_n(y), nodes y_j = cos(pi j / N);
// derivative recurrence c_m b_m = b_{m+2} + 2 (m+1) a_{m+1} (c_0 = 2).
#pragma once

#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "stage_launch.h"
#include "stage_scan.cuh"

namespace chdns {

// ---------------------------------------------------------------------------
// shared-memory views
// ---------------------------------------------------------------------------

// component r of a complex [n][ppc] tile: element n at p[n * stride]
template <typename T>
struct CompT {
  T* p;
  int stride;
  __device__ T& operator[](int n) const { return p[n * stride]; }
};
using CompS = CompT<double>;

// tau factor tables of one (mode, parity): element (f, i) at base[(f * Mh + i) * ppc]
struct TabSm {
  const double* base;
  int Mh, ppc;
  __device__ double e(int i) const { return base[(0 * Mh + i) * ppc]; }
  __device__ double h(int i) const { return base[(1 * Mh + i) * ppc]; }
  __device__ double b(int i) const { return base[(2 * Mh + i) * ppc]; }
  __device__ double Q(int i) const { return base[(3 * Mh + i) * ppc]; }
};

// folded tau tables of one (mode, parity) of a no-slip solve: element (f, i)
// at base[(f * Mh + i) * ppc], f = eA, eB, eC, h, b, W, and for the stage's
// Helmholtz operator E1 = (1 + alpha/beta) e
struct TabF {
  const double* base;
  int Mh, ppc;
  __device__ double eA(int i) const { return base[(0 * Mh + i) * ppc]; }
  __device__ double eB(int i) const { return base[(1 * Mh + i) * ppc]; }
  __device__ double eC(int i) const { return base[(2 * Mh + i) * ppc]; }
  __device__ double h(int i) const { return base[(3 * Mh + i) * ppc]; }
  __device__ double b(int i) const { return base[(4 * Mh + i) * ppc]; }
  __device__ double W(int i) const { return base[(5 * Mh + i) * ppc]; }
  __device__ double E1(int i) const { return base[(6 * Mh + i) * ppc]; }  // Helmholtz tables only
};
// a right-hand side value r and the operand x of a diagonal term E1_j x_j
struct RhsX {
  double r, x;
};

// ---------------------------------------------------------------------------
// Chebyshev-tau Dirichlet solve (D^2 - lam) f = r of one parity of one real
// component.  For n >= 2 the tau rows are equivalent to the quasi-tridiagonal
// rows
//   -lam cA_n f_{n-2} + (1 + lam cB_n) f_n - lam cC_n f_{n+2}
//       = cA_n r_{n-2} - cB_n r_n + cC_n r_{n+2},
//   cA_n = c_{n-2}/(4n(n-1)), cB_n = [n <= N-2]/(2(n^2-1)), cC_n = [n+2 <= N-2]/(4n(n+1)),
// obtained by integrating D^2 f = r + lam f twice; the two highest rows of r
// are dropped (tau).  With parity index i the rows i >= 1 are tridiagonal and
// the wall row sum_i f_i = s closes the system.  Bottom-up elimination gives
// f_i = a_i + b_i f_{i-1}; every f_i is then affine in f_0, which the wall row
// fixes.  The lam-dependent factors e = 1/den, h = U/den, b = -L/den, Q = prod b
// and 1/sum Q are precomputed per mode and stage.  rowc = [cA | cB | cC].
// ---------------------------------------------------------------------------
template <int MH, class Tab>
__device__ __forceinline__ void tau_seq(int N, int ny, int sig, const double (&r)[MH], double (&f)[MH],
                                        const Tab& T, double isq, double s, const double* __restrict__ rowc) {
  const int M = (N - sig) / 2 + 1;
  double anext = 0.0;
#pragma unroll
  for (int i = MH - 1; i >= 1; --i) {
    if (i < M) {
      const int n = 2 * i + sig;
      double R = fma_rn(-rowc[ny + n], r[i], mul_rn(rowc[n], r[i - 1]));
      if (i + 1 < MH && i + 1 < M) R = fma_rn(rowc[2 * ny + n], r[i + 1 < MH ? i + 1 : i], R);
      const double a = fma_rn(-T.h(i), anext, mul_rn(T.e(i), R));
      f[i] = a;
      anext = a;
    }
  }
  double Pp = 0.0, sum = 0.0;
#pragma unroll
  for (int i = 1; i < MH; ++i) {
    if (i < M) {
      Pp = fma_rn(T.b(i), Pp, f[i]);
      f[i] = Pp;
      sum += Pp;
    }
  }
  const double f0 = mul_rn(isq, s - sum);
  f[0] = f0;
#pragma unroll
  for (int i = 1; i < MH; ++i)
    if (i < M) f[i] = fma_rn(T.Q(i), f0, f[i]);
}

// symmetry class of a solve compiled for one class (a constant) or for both
template <int V>
__device__ __forceinline__ constexpr int class_of(std::integral_constant<int, V>) { return V; }
__device__ __forceinline__ int class_of(int v) { return v; }

// ---------------------------------------------------------------------------
// Free-slip top (open channel, top_bc = 1; paper Sec. 3.1).  The tau rows
// n >= 2 are those of the no-slip channel, so elimination still leaves each
// parity affine in its lowest coefficient, f = P + x Q (P_0 = 0, Q_0 = 1, Q
// the precomputed products of b); only the wall rows change, and they couple
// the two parities, which live in the two class threads of a mode:
//   omega_y, W:  f(-1) = S_e - S_o,  Df(+1) = S2_e + S2_o
//                (S = sum over the parity of f_n, S2 = sum of n^2 f_n);
//   U:           the same two rows and the flow rate, with the response to
//                the unknown forcing (even parity);
//   v:           v(+-1) stay Dirichlet per parity; phi = P + c vh per parity,
//                and D^2 v(+1) = A_e + A_o, Dv(-1) = -B_e + B_o
//                (A = sum n^2 (n^2 - 1) / 3 v_n, B = sum n^2 v_n) fix c_e, c_o.
// With the shifted unknowns f' = f + cc f_old every row's value is cc times
// that row applied to the old field.  Each thread of a pair publishes the
// sums of its parity; after a barrier both solve the same closure, summing
// in parity order, so both find the same coefficients.
// ---------------------------------------------------------------------------

// The affine family of one parity: f_i = P_i (i >= 1), f_0 = 0, with
// sp = sum P and sp2 = sum n^2 P (the same elimination as tau_seq).
template <int MH, class Tab>
__device__ __forceinline__ void tau_affine(int N, int ny, int sig, const double (&r)[MH], double (&f)[MH],
                                           const Tab& T, const double* __restrict__ rowc, double& sp, double& sp2) {
  const int M = (N - sig) / 2 + 1;
  double anext = 0.0;
#pragma unroll
  for (int i = MH - 1; i >= 1; --i) {
    if (i < M) {
      const int n = 2 * i + sig;
      double R = fma_rn(-rowc[ny + n], r[i], mul_rn(rowc[n], r[i - 1]));
      if (i + 1 < MH && i + 1 < M) R = fma_rn(rowc[2 * ny + n], r[i + 1 < MH ? i + 1 : i], R);
      const double a = fma_rn(-T.h(i), anext, mul_rn(T.e(i), R));
      f[i] = a;
      anext = a;
    }
  }
  double Pp = 0.0;
  sp = 0.0;
  sp2 = 0.0;
#pragma unroll
  for (int i = 1; i < MH; ++i) {
    if (i < M) {
      const double n = 2 * i + sig;
      Pp = fma_rn(T.b(i), Pp, f[i]);
      f[i] = Pp;
      sp += Pp;
      sp2 = fma_rn(n * n, Pp, sp2);
    }
  }
  f[0] = 0.0;
}

// f = P + x Q
template <int MH, class Arr, class Tab>
__device__ __forceinline__ void tau_close(int N, int sig, Arr& f, const Tab& T, double x) {
  const int M = (N - sig) / 2 + 1;
  f[0] = x;
#pragma unroll
  for (int i = 1; i < MH; ++i)
    if (i < M) f[i] = fma_rn(T.Q(i), x, f[i]);
}

// a11 x1 + a12 x2 = b1, a21 x1 + a22 x2 = b2 (Cramer's rule)
__device__ __forceinline__ void solve2(double a11, double a12, double a21, double a22, double b1, double b2,
                                       double* x1, double* x2) {
  const double id = 1.0 / fma_rn(a11, a22, -mul_rn(a12, a21));
  *x1 = mul_rn(fma_rn(b1, a22, -mul_rn(a12, b2)), id);
  *x2 = mul_rn(fma_rn(a11, b2, -mul_rn(a21, b1)), id);
}

// Dirichlet bottom and Neumann top rows over the two parities of omega_y or W.
// se, so: {sum P, sum n^2 P, sum f_old, sum n^2 f_old} of the even and odd
// parity; q*: the table sums sum Q and sum n^2 Q.
__device__ __forceinline__ void close_neumann_top(const double* se, const double* so, double qe, double qo,
                                                  double q2e, double q2o, double cc, double* xe, double* xo) {
  solve2(qe, -qo, q2e, q2o, fma_rn(cc, se[2] - so[2], -(se[0] - so[0])), fma_rn(cc, se[3] + so[3], -(se[1] + so[1])),
         xe, xo);
}

// Influence coefficients of v: se, so = {A_p, B_p, A_old, B_old}; a*, b*: A
// and B of the homogeneous solutions vh of the two parities.
__device__ __forceinline__ void close_free_slip_v(const double* se, const double* so, double ae, double ao,
                                                  double be, double bo, double cc, double* ce, double* co) {
  solve2(ae, ao, -be, bo, fma_rn(cc, se[2] + so[2], -(se[0] + so[0])), fma_rn(cc, so[3] - se[3], -(so[1] - se[1])),
         ce, co);
}

// Mean U at constant flow rate: unknowns (x_e, x_o, forcing).  se = {sum P,
// sum n^2 P, sum U_old, sum n^2 U_old, int P, int U_old}, so = the first four
// of the odd parity; q*: sum Q, sum n^2 Q; wq: int Q_e; u*: sum, sum n^2 and
// int of the forcing response (even).  int = sum of 2 / (1 - n^2) x_n.
__device__ __forceinline__ void close_free_slip_mean(const double* se, const double* so, double qe, double qo,
                                                     double q2e, double q2o, double wq, double us, double u2,
                                                     double uw, double cc, double flux, double* xe, double* xo,
                                                     double* fc) {
  const double a11 = qe, a12 = -qo, a13 = us;
  const double a21 = q2e, a22 = q2o, a23 = u2;
  const double a31 = wq, a32 = 0.0, a33 = uw;
  const double b1 = fma_rn(cc, se[2] - so[2], -(se[0] - so[0]));
  const double b2 = fma_rn(cc, se[3] + so[3], -(se[1] + so[1]));
  const double b3 = fma_rn(cc, se[5], flux) - se[4];
  // 2 x 2 minors (x y - z w, fused on the first product)
  auto det2 = [](double x, double y, double z, double w) { return fma_rn(x, y, -mul_rn(z, w)); };
  const double m1 = det2(a22, a33, a23, a32), m2 = det2(a21, a33, a23, a31), m3 = det2(a21, a32, a22, a31);
  const double id = 1.0 / fma_rn(a13, m3, fma_rn(a11, m1, -mul_rn(a12, m2)));
  *xe = mul_rn(fma_rn(a13, det2(b2, a32, a22, b3), fma_rn(b1, m1, -mul_rn(a12, det2(b2, a33, a23, b3)))), id);
  *xo = mul_rn(fma_rn(a13, det2(a21, b3, b2, a31), fma_rn(a11, det2(b2, a33, a23, b3), -mul_rn(b1, m2))), id);
  *fc = mul_rn(fma_rn(b1, m3, fma_rn(a11, det2(a22, b3, b2, a32), -mul_rn(a12, det2(a21, b3, b2, a31)))), id);
}

// Right-hand side of the v equation of parity sv and component r, one walk
// from n = N down to 0 carrying Dv, D^2 v, t = i kx H_x + i kz H_z and Dt;
// also stores h_v for the next stage.  Iteration i runs the other-parity step
// at 2i + sv + 1 (Dv, t) and then the own step at 2i + sv, so the register
// index i is fixed at compile time and the code is the same for both
// parities (threads of the two classes share warps).  The other-parity step
// at n = 0 (sv = 1) has no consumer and is not run.  The terms of v (Dv, D^2 v,
// phi) are FP64; the nonlinear-term part (t, Dt, h_v and dt (gamma h_v +
// zeta h_v')) runs in the node precision RN, FP32 in the mixed path, where
// H itself is FP32-accurate.  h_v' is read through HVr and the new h_v
// written through HVw (the same column, or a shared-memory copy and global).
template <int MH, typename RN>
__device__ __forceinline__ void v_walk(int N, int ny, int ppc, int sv, const CompS& Vc, const CompT<RN>& HVr,
                                       const CompT<RN>& HVw,
                                       const typename cpx<RN>::T* Hx, const typename cpx<RN>::T* Hy,
                                       const typename cpx<RN>::T* Hz, int r, double sgn, double kx, double kz,
                                       double k2, double cc, const StageCoef& sc, double (&rhs)[MH]) {
  using CN = typename cpx<RN>::T;
  const int ra = 1 - r;
  auto comp = [](const CN z, int qd) { return qd == 0 ? z.x : z.y; };
  const double dsv = 2.0 * sv;
  const RN dsvn = (RN)(2 * sv);
  const RN sgnn = (RN)sgn, kxn = (RN)kx, kzn = (RN)kz, k2n = (RN)k2;
  const RN dtn = (RN)sc.dt, gan = (RN)sc.gamma, zen = (RN)sc.zeta;
  double dv = 0.0, d2v = 0.0;
  RN tt = 0, dtt = 0;
#pragma unroll
  for (int i = MH - 1; i >= 0; --i) {
    const int no = 2 * i + sv + 1;
    if (no <= N) {
      const double vn1 = (no + 1 <= N) ? Vc[no + 1] : 0.0;
      dv = fma_rn((double)(4 * i + 4) + dsv, vn1, dv);  // 2 (no + 1)
      tt = mul_rn(sgnn, fma_rn(kxn, comp(Hx[no * ppc], ra), mul_rn(kzn, comp(Hz[no * ppc], ra))));
    }
    const int n = 2 * i + sv;
    if (n <= N) {
      const double fac = (double)(4 * i + 2) + dsv;  // 2 (n + 1)
      const RN facn = (RN)(4 * i + 2) + dsvn;
      const double t1 = fma_rn(fac, dv, d2v);
      const RN t2 = fma_rn(facn, (n + 1 <= N) ? tt : (RN)0, dtt);
      d2v = (n == 0) ? 0.5 * t1 : t1;
      dtt = (n == 0) ? (RN)0.5 * t2 : t2;
      const double phi = fma_rn(-k2, Vc[n], d2v);
      const RN hv = fma_rn(-k2n, comp(Hy[n * ppc], r), -dtt);
      const RN hp = HVr[n];
      HVw[n] = hv;
      const RN q = mul_rn(dtn, fma_rn(gan, hv, mul_rn(zen, hp)));
      rhs[i] = fma_rn(1.0 + cc, phi, (double)q);
    }
  }
}

// ---------------------------------------------------------------------------
// The implicit solves of the no-slip channel with one register array per
// thread.  tau_fused is tau_seq with the right-hand side produced on the fly:
// rhs(i) is called once per coefficient, for i = M-1 down to 0, and row i of
// the elimination runs as soon as r_{i-1} exists, so no array of right-hand
// sides is held.  A solve may read its right-hand side from f itself (the
// second solve of v): f[i] is read at step i and written at step i - 1.
// The wall value s is asked for after the last call of rhs, so the sums that
// rhs accumulates are complete.  The row arithmetic is tau_seq's.  f is a
// per-thread array of MH doubles: registers (RegArr), or a column of shared
// memory (SmemArr) where MH doubles per thread exceed the register file.
// ---------------------------------------------------------------------------
template <int MH, class V = double>
struct RegArr {
  V v[MH];
  __device__ __forceinline__ V& operator[](int i) { return v[i]; }
};
struct SmemArr {
  double* p;
  int stride;
  __device__ __forceinline__ double& operator[](int i) const { return p[i * stride]; }
};

template <int MH, class Arr, class Tab, class Rhs, class Wall>
__device__ __forceinline__ void tau_fused(int N, int ny, int sig, Rhs&& rhs, Arr& f, const Tab& T, double isq,
                                          Wall&& wall, const double* __restrict__ rowc) {
  using V = std::decay_t<decltype(f[0])>;  // double, or a Pair of components
  const int M = (N - sig) / 2 + 1;
  V r1{}, r2{}, anext{};  // r_{i+1}, r_{i+2}, a_{i+2}
#pragma unroll
  for (int i = MH - 1; i >= 0; --i) {
    V r0{};
    if (i < M) r0 = rhs(i);
    const int j = i + 1;  // row j needs r_{j-1} = r0, r_j = r1, r_{j+1} = r2
    if (j < MH && j < M) {
      const int n = 2 * j + sig;
      V R = fma_rn(-rowc[ny + n], r1, mul_rn(rowc[n], r0));
      if (j + 1 < M) R = fma_rn(rowc[2 * ny + n], r2, R);
      const V a = fma_rn(-T.h(j), anext, mul_rn(T.e(j), R));
      f[j] = a;
      anext = a;
    }
    r2 = r1;
    r1 = r0;
  }
  V Pp{}, sum{};
#pragma unroll
  for (int i = 1; i < MH; ++i) {
    if (i < M) {
      Pp = fma_rn(T.b(i), Pp, f[i]);
      f[i] = Pp;
      sum = sum + Pp;
    }
  }
  const V f0 = mul_rn(isq, wall() - sum);
  f[0] = f0;
#pragma unroll
  for (int i = 1; i < MH; ++i)
    if (i < M) f[i] = fma_rn(T.Q(i), f0, f[i]);
}

// tau_fused on the folded tables (no-slip top).  Row j of the elimination
// is a_j = eA_j r_{j-1} - eB_j r_j + eC_j r_{j+1} - h_j a_{j+1}: the same
// rows with the factor e taken into the row constants.  The wall row needs
// sum_i P_i, the sum of the particular solution P_i = a_i + b_i P_{i-1}
// (P_0 = 0); it equals sum_i W_i a_i and is accumulated during the
// elimination.  f_0 = (s - sum_i P_i) / sum_i Q_i then follows at once, and the
// back substitution f_i = a_i + b_i f_{i-1} gives the solution in one pass
// (f_i = P_i + Q_i f_0, Q_i the products of b).  With DIAG, rhs(i) returns
// RhsX{r_i, x_i} and row j takes the extra term E1_j x_j.
template <int MH, bool DIAG = false, class Arr, class Rhs, class Wall>
__device__ __forceinline__ void tau_fold(int N, int sig, Rhs&& rhs, Arr& f, const TabF& T, double isq,
                                         Wall&& wall) {
  const int M = (N - sig) / 2 + 1;
  double r1 = 0.0, r2 = 0.0, x1 = 0.0, anext = 0.0, sum = 0.0;  // r_{i+1}, r_{i+2}, x_{i+1}, a_{i+2}
#pragma unroll
  for (int i = MH - 1; i >= 0; --i) {
    double r0 = 0.0, x0 = 0.0;
    if (i < M) {
      if constexpr (DIAG) {
        const RhsX v = rhs(i);
        r0 = v.r;
        x0 = v.x;
      } else {
        r0 = rhs(i);
      }
    }
    const int j = i + 1;  // row j needs r_{j-1} = r0, r_j = r1, r_{j+1} = r2 (and x_j = x1)
    if (j < MH && j < M) {
      double R = fma_rn(-T.eB(j), r1, mul_rn(T.eA(j), r0));
      if (j + 1 < M) R = fma_rn(T.eC(j), r2, R);
      if constexpr (DIAG) R = fma_rn(T.E1(j), x1, R);
      const double a = fma_rn(-T.h(j), anext, R);
      f[j] = a;
      anext = a;
      sum = fma_rn(T.W(j), a, sum);
    }
    r2 = r1;
    r1 = r0;
    x1 = x0;
  }
  double fp = mul_rn(isq, wall() - sum);
  f[0] = fp;
#pragma unroll
  for (int i = 1; i < MH; ++i)
    if (i < M) {
      fp = fma_rn(T.b(i), fp, f[i]);
      f[i] = fp;
    }
}

// omega_y of parity sq: (D^2 - lam) g' = -((1 + cc) g + dt (gamma h_g + zeta
// h_g'))/(beta dt nu), the factor -1/(beta dt nu) folded into the table's e;
// wall row sum g' = cc sum g; g <- g' - cc g.  h_g = sgn (-kx H_z + kz H_x) of
// the other component, in the node precision; h_g' is read through HGr and
// the new h_g written through HGw.
template <int MH, typename RN, class Arr, class GV, class HR, class HW, class Tab>
__device__ __forceinline__ void omega_solve(Arr& f, int N, int ny, int ppc, int sq, const GV& Gc, const HR& HGr,
                                            const HW& HGw, const typename cpx<RN>::T* Hx,
                                            const typename cpx<RN>::T* Hz, int r, double sgn, double kx, double kz,
                                            double cc, const StageCoef& sc, const Tab& T, double isq) {
  using CN = typename cpx<RN>::T;
  const int ra = 1 - r;
  auto comp = [](const CN z, int qd) { return qd == 0 ? z.x : z.y; };
  const RN sgnn = (RN)sgn, kxn = (RN)kx, kzn = (RN)kz;
  const RN dtn = (RN)sc.dt, gan = (RN)sc.gamma, zen = (RN)sc.zeta;
  const int M = (N - sq) / 2 + 1;
  double sum = 0.0;
  tau_fold<MH>(
      N, sq,
      [&](int i) {
        const int n = 2 * i + sq;
        const double gn = Gc[n];
        const RN hg = mul_rn(sgnn, fma_rn(-kxn, comp(Hz[n * ppc], ra), mul_rn(kzn, comp(Hx[n * ppc], ra))));
        const RN hp = HGr[n];
        HGw[n] = hg;
        const RN q = mul_rn(dtn, fma_rn(gan, hg, mul_rn(zen, hp)));
        sum += gn;
        return fma_rn(1.0 + cc, gn, (double)q);
      },
      f, T, isq, [&] { return mul_rn(cc, sum); });
#pragma unroll
  for (int i = 0; i < MH; ++i)
    if (i < M) {
      const int n = 2 * i + sq;
      Gc[n] = fma_rn(-cc, Gc[n], f[i]);
    }
}

// v of parity sv.  The phi solve's right-hand side is (1 + cc)(D^2 v - k^2 v)
// + q; its tau rows apply to it the stencil r -> cA r_{n-2} - cB r_n +
// cC r_{n+2}, which integrates D^2 twice, so the stencil of D^2 v is v_n
// itself (n >= 2).  Row j therefore takes (1 + cc) e v_n through E1 plus the
// stencil of u = -(1 + cc) k^2 v + q, and no D^2 v is formed; only the FP32
// walk of t and Dt (from n = N down) remains for q.  The wall sums S0 = sum v,
// S2 = sum n^2 v of the old field are taken on the way down.  Then the Dirichlet solve of
// (D^2 - k^2) v_p = phi with v_p(+-1) = cc v(+-1) + (wall velocity), reading
// phi from the same array, and the influence correction c_I vh that fixes
// Dv at the wall: v <- v_p + c_I vh - cc v.
template <int MH, typename RN, class Arr, class VV, class HR, class HW, class Tab, class TabP, class VH>
__device__ __forceinline__ void v_solve(Arr& f, int N, int ny, int ppc, int sv, const VV& Vc, const HR& HVr,
                                        const HW& HVw,
                                        const typename cpx<RN>::T* Hx, const typename cpx<RN>::T* Hy,
                                        const typename cpx<RN>::T* Hz, int r, double sgn, double kx, double kz,
                                        double k2, double cc, const StageCoef& sc, const Tab& Th, double isq_h,
                                        const TabP& Tp, double isq_p, const VH& vh, double idv, double vw) {
  using CN = typename cpx<RN>::T;
  const int ra = 1 - r;
  auto comp = [](const CN z, int qd) { return qd == 0 ? z.x : z.y; };
  const RN dsvn = (RN)(2 * sv);
  const RN sgnn = (RN)sgn, kxn = (RN)kx, kzn = (RN)kz, k2n = (RN)k2;
  const RN dtn = (RN)sc.dt, gan = (RN)sc.gamma, zen = (RN)sc.zeta;
  const int M = (N - sv) / 2 + 1;
  const double ck2 = -(1.0 + cc) * k2;
  double S0 = 0.0, S2 = 0.0;
  RN tt = 0, dtt = 0;
  tau_fold<MH, true>(
      N, sv,
      [&](int i) {
        const int no = 2 * i + sv + 1;
        if (no <= N) tt = mul_rn(sgnn, fma_rn(kxn, comp(Hx[no * ppc], ra), mul_rn(kzn, comp(Hz[no * ppc], ra))));
        const int n = 2 * i + sv;
        const RN facn = (RN)(4 * i + 2) + dsvn;  // 2 (n + 1)
        const RN t2 = fma_rn(facn, (n + 1 <= N) ? tt : (RN)0, dtt);
        dtt = (n == 0) ? (RN)0.5 * t2 : t2;
        const double vn = Vc[n];
        S0 += vn;
        S2 = fma_rn((double)n * n, vn, S2);
        const RN hv = fma_rn(-k2n, comp(Hy[n * ppc], r), -dtt);
        const RN hp = HVr[n];
        HVw[n] = hv;
        const RN q = mul_rn(dtn, fma_rn(gan, hv, mul_rn(zen, hp)));
        return RhsX{fma_rn(ck2, vn, (double)q), vn};
      },
      f, Th, isq_h, [] { return 0.0; });
  const double s = fma_rn(cc, S0, ((sv == 0) ? 0.5 : -0.5) * vw);
  tau_fold<MH>(N, sv, [&](int i) { return f[i]; }, f, Tp, isq_p, [&] { return s; });
  double dp = 0.0;
#pragma unroll
  for (int i = 0; i < MH; ++i)
    if (i < M) {
      const double n = 2 * i + sv;
      dp = fma_rn(n * n, f[i], dp);
    }
  const double cI = mul_rn(fma_rn(cc, S2, -dp), idv);
#pragma unroll
  for (int i = 0; i < MH; ++i)
    if (i < M) {
      const int n = 2 * i + sv;
      Vc[n] = fma_rn(-cc, Vc[n], fma_rn(cI, vh(i), f[i]));
    }
}

// ---------------------------------------------------------------------------
// The affine families of the free-slip top with the right-hand sides produced
// on the fly, as in tau_fused.  tau_affine_fused leaves f_i = P_i (i >= 1),
// f_0 = 0, with sp = sum P and sp2 = sum n^2 P; tau_close then adds x Q.
// The wall sums of the old field are taken on the way down.
// ---------------------------------------------------------------------------
template <int MH, class Arr, class Tab, class Rhs>
__device__ __forceinline__ void tau_affine_fused(int N, int ny, int sig, Rhs&& rhs, Arr& f, const Tab& T,
                                                 const double* __restrict__ rowc, double& sp, double& sp2) {
  const int M = (N - sig) / 2 + 1;
  double r1 = 0.0, r2 = 0.0, anext = 0.0;
#pragma unroll
  for (int i = MH - 1; i >= 0; --i) {
    double r0 = 0.0;
    if (i < M) r0 = rhs(i);
    const int j = i + 1;
    if (j < MH && j < M) {
      const int n = 2 * j + sig;
      double R = fma_rn(-rowc[ny + n], r1, mul_rn(rowc[n], r0));
      if (j + 1 < M) R = fma_rn(rowc[2 * ny + n], r2, R);
      const double a = fma_rn(-T.h(j), anext, mul_rn(T.e(j), R));
      f[j] = a;
      anext = a;
    }
    r2 = r1;
    r1 = r0;
  }
  double Pp = 0.0;
  sp = 0.0;
  sp2 = 0.0;
#pragma unroll
  for (int i = 1; i < MH; ++i) {
    if (i < M) {
      const double n = 2 * i + sig;
      Pp = fma_rn(T.b(i), Pp, f[i]);
      f[i] = Pp;
      sp += Pp;
      sp2 = fma_rn(n * n, Pp, sp2);
    }
  }
  f[0] = 0.0;
}

// omega_y of parity sq under the free-slip top: the affine family and
// out = {sum P, sum n^2 P, sum g, sum n^2 g} for the closure
template <int MH, typename RN, class Arr, class GV, class HR, class HW, class Tab>
__device__ __forceinline__ void omega_open_affine(Arr& f, int N, int ny, int ppc, int sq, const GV& Gc,
                                                  const HR& HGr, const HW& HGw, const typename cpx<RN>::T* Hx,
                                                  const typename cpx<RN>::T* Hz, int r, double sgn, double kx,
                                                  double kz, double cc, const StageCoef& sc, const Tab& T,
                                                  const double* __restrict__ rowc, double* out) {
  using CN = typename cpx<RN>::T;
  const int ra = 1 - r;
  auto comp = [](const CN z, int qd) { return qd == 0 ? z.x : z.y; };
  const RN sgnn = (RN)sgn, kxn = (RN)kx, kzn = (RN)kz;
  const RN dtn = (RN)sc.dt, gan = (RN)sc.gamma, zen = (RN)sc.zeta;
  double so = 0.0, so2 = 0.0, sp, sp2;
  tau_affine_fused<MH>(
      N, ny, sq,
      [&](int i) {
        const int n = 2 * i + sq;
        const double gn = Gc[n];
        const RN hg = mul_rn(sgnn, fma_rn(-kxn, comp(Hz[n * ppc], ra), mul_rn(kzn, comp(Hx[n * ppc], ra))));
        const RN hp = HGr[n];
        HGw[n] = hg;
        const RN q = mul_rn(dtn, fma_rn(gan, hg, mul_rn(zen, hp)));
        so += gn;
        so2 = fma_rn((double)n * n, gn, so2);
        return fma_rn(1.0 + cc, gn, (double)q);
      },
      f, T, rowc, sp, sp2);
  out[0] = sp;
  out[1] = sp2;
  out[2] = so;
  out[3] = so2;
}

// mean flow of parity s under the free-slip top (U: e = 0, W: e = 1): the
// affine family and out = {sum P, sum n^2 P, sum X, sum n^2 X, int P, int X}
// (int x = sum 2 / (1 - n^2) x_n, even parity only)
template <int MH, typename RN, class Arr, class Tab>
__device__ __forceinline__ void mean_open_affine(Arr& f, int N, int ny, int ppc, int s, double* X, double* XP,
                                                 const typename cpx<RN>::T* Hm, double cc, const StageCoef& sc,
                                                 const Tab& T, const double* __restrict__ rowc, double* out) {
  const int M = (N - s) / 2 + 1;
  double so = 0.0, so2 = 0.0, wo = 0.0, sp, sp2;
  tau_affine_fused<MH>(
      N, ny, s,
      [&](int i) {
        const int n = 2 * i + s;
        const double xn = X[n];
        const double hv = (double)Hm[n * ppc].x;
        const double hp = XP[n];
        XP[n] = hv;
        so += xn;
        so2 = fma_rn((double)n * n, xn, so2);
        if (s == 0) wo = fma_rn(2.0 / (1.0 - (double)n * n), xn, wo);
        return fma_rn(1.0 + cc, xn, mul_rn(sc.dt, fma_rn(sc.gamma, hv, mul_rn(sc.zeta, hp))));
      },
      f, T, rowc, sp, sp2);
  double wp = 0.0;
  if (s == 0) {
#pragma unroll
    for (int i = 0; i < MH; ++i)
      if (i < M) wp = fma_rn(2.0 / (1.0 - 4.0 * (double)i * i), f[i], wp);
  }
  out[0] = sp;
  out[1] = sp2;
  out[2] = so;
  out[3] = so2;
  out[4] = wp;
  out[5] = wo;
}

// v of parity sv under the free-slip top: phi and v_p with the Dirichlet rows
// of the no-slip channel (f = v_p on return), then out = {A_p, B_p, A_old,
// B_old} of the free-slip rows (A = sum n^2 (n^2 - 1) / 3 v_n, B = sum n^2
// v_n); vw is the wall velocity of this component
template <int MH, typename RN, class Arr, class VV, class HR, class HW, class Tab, class TabP>
__device__ __forceinline__ void v_open_part(Arr& f, int N, int ny, int ppc, int sv, const VV& Vc, const HR& HVr,
                                            const HW& HVw, const typename cpx<RN>::T* Hx,
                                            const typename cpx<RN>::T* Hy, const typename cpx<RN>::T* Hz, int r,
                                            double sgn, double kx, double kz, double k2, double cc,
                                            const StageCoef& sc, const Tab& Th, double isq_h, const TabP& Tp,
                                            double isq_p, double vw, const double* __restrict__ rowc, double* out) {
  using CN = typename cpx<RN>::T;
  const int ra = 1 - r;
  auto comp = [](const CN z, int qd) { return qd == 0 ? z.x : z.y; };
  const double dsv = 2.0 * sv;
  const RN dsvn = (RN)(2 * sv);
  const RN sgnn = (RN)sgn, kxn = (RN)kx, kzn = (RN)kz, k2n = (RN)k2;
  const RN dtn = (RN)sc.dt, gan = (RN)sc.gamma, zen = (RN)sc.zeta;
  const int M = (N - sv) / 2 + 1;
  double dv = 0.0, d2v = 0.0, S0 = 0.0, Bo = 0.0, Ao = 0.0;
  RN tt = 0, dtt = 0;
  tau_fused<MH>(
      N, ny, sv,
      [&](int i) {
        const int no = 2 * i + sv + 1;
        if (no <= N) {
          const double vn1 = (no + 1 <= N) ? Vc[no + 1] : 0.0;
          dv = fma_rn((double)(4 * i + 4) + dsv, vn1, dv);  // 2 (no + 1)
          tt = mul_rn(sgnn, fma_rn(kxn, comp(Hx[no * ppc], ra), mul_rn(kzn, comp(Hz[no * ppc], ra))));
        }
        const int n = 2 * i + sv;
        const double fac = (double)(4 * i + 2) + dsv;  // 2 (n + 1)
        const RN facn = (RN)(4 * i + 2) + dsvn;
        const double t1 = fma_rn(fac, dv, d2v);
        const RN t2 = fma_rn(facn, (n + 1 <= N) ? tt : (RN)0, dtt);
        d2v = (n == 0) ? 0.5 * t1 : t1;
        dtt = (n == 0) ? (RN)0.5 * t2 : t2;
        const double vn = Vc[n];
        const double nn = (double)n * n;
        S0 += vn;
        Bo = fma_rn(nn, vn, Bo);
        Ao = fma_rn(nn * (nn - 1.0) / 3.0, vn, Ao);
        const double phi = fma_rn(-k2, vn, d2v);
        const RN hv = fma_rn(-k2n, comp(Hy[n * ppc], r), -dtt);
        const RN hp = HVr[n];
        HVw[n] = hv;
        const RN q = mul_rn(dtn, fma_rn(gan, hv, mul_rn(zen, hp)));
        return fma_rn(1.0 + cc, phi, (double)q);
      },
      f, Th, isq_h, [] { return 0.0; }, rowc);
  const double s = fma_rn(cc, S0, ((sv == 0) ? 0.5 : -0.5) * vw);
  tau_fused<MH>(N, ny, sv, [&](int i) { return f[i]; }, f, Tp, isq_p, [&] { return s; }, rowc);
  double Ap = 0.0, Bp = 0.0;
#pragma unroll
  for (int i = 0; i < MH; ++i)
    if (i < M) {
      const double n = 2 * i + sv;
      Bp = fma_rn(n * n, f[i], Bp);
      Ap = fma_rn(n * n * (n * n - 1.0) / 3.0, f[i], Ap);
    }
  out[0] = Ap;
  out[1] = Bp;
  out[2] = Ao;
  out[3] = Bo;
}

// mean flow of parity s: U (e = 0, at constant flow rate through the
// response u1 to a unit forcing) or W (e = 1); X the coefficients, XP the
// previous plane means of H_x or H_z (FP64), Hm the new plane mean.
template <int MH, typename RN, class Arr, class Tab>
__device__ __forceinline__ void mean_solve(Arr& f, int N, int ny, int ppc, int s, int e, double* X, double* XP,
                                           const typename cpx<RN>::T* Hm, double cc, const StageCoef& sc,
                                           const Tab& T, double isq,
                                           const double* __restrict__ u1, double u1_iflux) {
  const int M = (N - s) / 2 + 1;
  double sum = 0.0, flux_old = 0.0;
  tau_fold<MH>(
      N, s,
      [&](int i) {
        const int n = 2 * i + s;
        const double xn = X[n];
        const double hv = (double)Hm[n * ppc].x;
        const double hp = XP[n];
        XP[n] = hv;
        sum += xn;
        if (s == 0) flux_old = fma_rn(2.0 / (1.0 - (double)n * n), xn, flux_old);
        return fma_rn(1.0 + cc, xn, mul_rn(sc.dt, fma_rn(sc.gamma, hv, mul_rn(sc.zeta, hp))));
      },
      f, T, isq, [&] { return mul_rn(cc, sum); });
  double fc = 0.0;
  if (e == 0 && s == 0) {
    double flux = 0.0;
#pragma unroll
    for (int i = 0; i < MH; ++i)
      if (i < M) flux = fma_rn(2.0 / (1.0 - 4.0 * (double)i * i), f[i], flux);
    fc = mul_rn(fma_rn(cc, flux_old, sc.flux) - flux, u1_iflux);
  }
#pragma unroll
  for (int i = 0; i < MH; ++i) {
    if (i < M) {
      const int n = 2 * i + s;
      double v = fma_rn(-cc, X[n], f[i]);
      if (e == 0 && s == 0) v = fma_rn(fc, u1[i], v);
      X[n] = v;
    }
  }
}


// One (mode p, class, component r) thread's implicit solves under the no-slip
// top: the mean flow (p = 0), else omega_y of parity 1 - c and v of parity c.
// H_x, H_y, H_z: Chebyshev coefficients of the mode, element n at n * hs;
// HGr, HVr: the previous nonlinear right-hand sides (node precision); the new
// ones go to the pencil buffers.  Each solve keeps its array of MH doubles in
// registers (col = nullptr) or in the thread's column of shared memory,
// col[i * cs].
template <int MH, typename RN, bool SMEM, class Cls>
__device__ __forceinline__ void post_solve_noslip(double* col, int cs, Cls cls, const Grid& g, const PencilBufs& pb,
                                                  const DevTables& t, const StageCoef& sc, int b, int p, int r,
                                                  const typename cpx<RN>::T* Hx, const typename cpx<RN>::T* Hy,
                                                  const typename cpx<RN>::T* Hz, int hs, const CompT<RN>& HGr,
                                                  const CompT<RN>& HVr) {
  const int c = class_of(cls);
  const int P = g.P, ny = g.ny, N = g.N, Mh = t.tau.Mh;
  const double cc = sc.alpha / sc.beta;
  auto comp = [](auto z, int qq) { return qq == 0 ? z.x : z.y; };
  auto helm = [&](int sig) { return TabF{t.tau.helm_f + (size_t)(sc.k * 2 + sig) * 7 * Mh * P + p, Mh, P}; };
  auto helm_isq = [&](int sig) { return t.tau.helm_isq[(size_t)(sc.k * 2 + sig) * P + p]; };
  if (p == 0) {
    // mean mode: U (r = 0) at constant flow rate and W (r = 1), parity c
    const int e = r;
    auto run = [&](auto& f) {
      mean_solve<MH, RN>(f, N, ny, hs, c, e, (e == 0 ? pb.UM : pb.WM) + (size_t)b * ny,
                       (e == 0 ? pb.HXP : pb.HZP) + (size_t)b * ny, (e == 0) ? Hx : Hz, cc, sc, helm(c),
                       helm_isq(c), t.tau.u1 + (size_t)sc.k * Mh, t.tau.u1_iflux[sc.k]);
    };
    if constexpr (SMEM) {
      SmemArr f{col, cs};
      run(f);
    } else {
      RegArr<MH> f;
      run(f);
    }
    return;
  }
  const int row = p / g.nxh, ix = p % g.nxh;
  const double kx = t.kx[ix], kz = t.kz[row], k2 = kx * kx + kz * kz;
  const double sgn = (r == 0) ? -1.0 : 1.0;
  const size_t base = 2 * ((size_t)b * ny * P + p) + r;  // component r of element n at base + 2 P n
  {
    // wall-normal vorticity, parity 1 - c; previous right-hand sides are
    // stored in the node precision
    const int sq = 1 - c;
    const CompS Gc{reinterpret_cast<double*>(pb.G) + base, 2 * P};
    const CompT<RN> HGc{reinterpret_cast<RN*>(pb.HGP) + base, 2 * P};
    auto run = [&](auto& f) {
      omega_solve<MH, RN>(f, N, ny, hs, sq, Gc, HGr, HGc, Hx, Hz, r, sgn, kx, kz, cc, sc, helm(sq), helm_isq(sq));
    };
    if constexpr (SMEM) {
      SmemArr f{col, cs};
      run(f);
    } else {
      RegArr<MH> f;
      run(f);
    }
  }
  {
    // wall-normal velocity, parity c
    const int sv = c;
    const CompS Vc{reinterpret_cast<double*>(pb.V) + base, 2 * P};
    const CompT<RN> HVc{reinterpret_cast<RN*>(pb.HVP) + base, 2 * P};
    const size_t vo = (size_t)b * P + p;
    const double vw = fma_rn(sc.theta, comp(pb.vw_new[vo], r) - comp(pb.vw_old[vo], r), comp(pb.vw_old[vo], r));
    const TabF TP{t.tau.pois_f + (size_t)sv * 6 * Mh * P + p, Mh, P};
    const double* vh = t.tau.vh + (size_t)(sc.k * 2 + sv) * Mh * P + p;
    auto run = [&](auto& f) {
      v_solve<MH, RN>(f, N, ny, hs, sv, Vc, HVr, HVc, Hx, Hy, Hz, r, sgn, kx, kz, k2, cc, sc, helm(sv),
                      helm_isq(sv), TP, t.tau.pois_isq[(size_t)sv * P + p], [&](int i) { return vh[(size_t)i * P]; },
                      t.tau.vh_idv[(size_t)(sc.k * 2 + sv) * P + p], vw);
    };
    if constexpr (SMEM) {
      SmemArr f{col, cs};
      run(f);
    } else {
      RegArr<MH> f;
      run(f);
    }
  }
}

// cos(pi j n / N) table in the node precision
template <typename RN>
__device__ __forceinline__ const RN* cheb_table(const DevTables& t);
template <>
__device__ __forceinline__ const double* cheb_table<double>(const DevTables& t) { return t.cheb; }
template <>
__device__ __forceinline__ const float* cheb_table<float>(const DevTables& t) { return t.cheb_f; }

// Chebyshev coefficients a_n, n = n0 + dn k (k < KN, all of one parity), of
// one field of one mode from its nodal values col[j * stride], j = 0..N, by the
// direct sums a_n = (2 / (N c_n)) sum_j'' f_j cos(pi j n / N) over the folded
// pairs f_j + (-1)^n f_{N-j} (sg = (-1)^n), accumulated over j in ascending
// order; c_0 = c_N = 2, the end nodes weigh 1/2.
template <typename RN, int KN>
__device__ __forceinline__ void analysis_sums(const typename cpx<RN>::T* col, int stride, int N, int ny,
                                              const RN* __restrict__ cheb, int n0, int dn, RN sg,
                                              typename cpx<RN>::T (&acc)[KN]) {
  using CN = typename cpx<RN>::T;
  CN a[KN];
  const CN w0 = (RN)0.5 * (col[0] + sg * col[N * stride]);  // j = 0 and j = N weigh 1/2
#pragma unroll
  for (int k = 0; k < KN; ++k) a[k] = w0;
  for (int j = 1; 2 * j < N; ++j) {
    const CN fold = col[j * stride] + sg * col[(N - j) * stride];
#pragma unroll
    for (int k = 0; k < KN; ++k) {
      const int n = n0 + dn * k;
      a[k] = a[k] + cheb[(size_t)min(n, N) * ny + j] * fold;
    }
  }
  const RN s0 = (RN)2.0 / (RN)N;
#pragma unroll
  for (int k = 0; k < KN; ++k) {
    const int n = n0 + dn * k;
    const RN cbn = (n == 0 || n == N) ? (RN)2.0 : (RN)1.0;
    CN v = a[k];
    if ((N & 1) == 0) v = v + cheb[(size_t)min(n, N) * ny + N / 2] * col[(N / 2) * stride];
    acc[k] = (s0 / cbn) * v;
  }
}

template <typename C> __device__ __forceinline__ C to_node(double2 v);
template <> __device__ __forceinline__ double2 to_node<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 to_node<float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }

// ---------------------------------------------------------------------------
// Fast Chebyshev synthesis (DCT-I) of complex lines through an N-point FFT,
// N even:  F_j = sum_{n=0}^{N} x_n cos(pi j n / N), j = 0..N.
// With y_n = (x_n + x_{N-n})/2 - sin(pi n / N) (x_n - x_{N-n}), n = 0..N-1,
// and Z_k = sum_n y_n e^{2 pi i k n / N}: the cosine sums pick out the part
// of y symmetric under n -> N - n, which reproduces the even outputs, and the
// sine sums the antisymmetric part, which gives differences of odd outputs:
//   F_{2k} = (Z_k + Z_{N-k}) / 2 + (x_0 + x_N) / 2,          k = 0..N/2,
//   F_{2k+1} = F_{2k-1} - i (Z_k - Z_{N-k}) / 2,             k = 1..N/2-1,
//   F_1 = sum_n x_n cos(pi n / N).
// O(N log N) FP64 operations per line instead of the (N/2)(N+1) of the sums.
// Lines: line l = f G + pl at buf + f LS + pl, element stride G.
// ---------------------------------------------------------------------------
template <int N, int ST>
__device__ __forceinline__ void lines_dif(double2* buf, const double2* tw, int nlines, int G, int LS) {
  if constexpr (ST < ct_nst(N)) {
    constexpr int r = ct_radix(N, ST);
    constexpr int L = ct_len_before(N, ST);
    constexpr int m = L / r;
    constexpr int nb = N / r;
    constexpr int tstep = N / L;
    for (int w = threadIdx.x; w < nlines * nb; w += blockDim.x) {
      const int l = w % nlines, bf = w / nlines;
      double2* base = buf + (l / G) * LS + (l % G);
      const int blk = bf / m, q = bf % m;
      const int i0 = blk * L + q;
      double2 x[r];
#pragma unroll
      for (int t = 0; t < r; ++t) x[t] = base[(i0 + t * m) * G];
      small_dft_ct<+1, r, double2, double>(x);
#pragma unroll
      for (int u = 0; u < r; ++u) {
        double2 y = x[u];
        if (u > 0 && q > 0) y = cmul_rn(y, tw[q * u * tstep]);
        base[(i0 + u * m) * G] = y;
      }
    }
    __syncthreads();
    lines_dif<N, ST + 1>(buf, tw, nlines, G, LS);
  }
}

// position of frequency k in the digit-reversed output of the DIF passes:
// sum over passes of (digit of k in that pass's radix) x (sub-block length)
template <int N>
__device__ __forceinline__ int dif_pos(int k) {
  int p = 0, L = N;
#pragma unroll
  for (int st = 0; st < ct_nst(N); ++st) {
    const int r = ct_radix(N, st);
    const int m = L / r;
    p += (k % r) * m;
    k /= r;
    L = m;
  }
  return p;
}

// Chebyshev analysis of the three fields of a tile in FP64 through the same
// FFT form of the DCT-I: a_n = (2 / (N cb_n)) F_n, F the DCT-I of
// g_j = f_j / cb_j (cb_0 = cb_N = 2).  X: tile [3][ny][ppc], nodal values in,
// coefficients out.  The FFT leaves Z in digit-reversed order in the tile's
// own storage: each even output is stored in Z_k's slot and each odd-output
// difference in Z_{N-k}'s slot (every slot read and written by one item
// only), and the natural-order coefficients pass through this tile's columns
// of the global node array Rt (modes of this CTA, read by no other CTA) before
// they are copied back.  hf: shared scratch of 6 ppc values.
template <int NF>
__device__ __forceinline__ void analysis_fft(double2* X, int ppc, int ny, int P, int p0, double2* hf,
                                             const double* cheb, const double2* tw, double2* Rt) {
  constexpr int N = NF;
  const int nl = 3 * ppc, LS = ny * ppc;
  const int tid = threadIdx.x, nt = blockDim.x;
  double2* sHalf = hf;       // (g_0 + g_N) / 2
  double2* sF1 = hf + nl;    // F_1
  for (int l = tid; l < nl; l += nt) {
    double2* x = X + (l / ppc) * LS + (l % ppc);
    x[0] = 0.5 * x[0];
    x[N * ppc] = 0.5 * x[N * ppc];
    double2 s1 = mk(0.0, 0.0);
    for (int n = 0; n <= N; ++n) s1 = s1 + cheb[ny + n] * x[n * ppc];
    sF1[l] = s1;
    sHalf[l] = 0.5 * (x[0] + x[N * ppc]);
  }
  __syncthreads();
  for (int w = tid; w < nl * (N / 2); w += nt) {
    const int l = w % nl, n = w / nl;
    double2* x = X + (l / ppc) * LS + (l % ppc);
    if (n == 0) {
      x[0] = sHalf[l];
      continue;
    }
    const double2 xa = x[n * ppc], xb = x[(N - n) * ppc];
    const double sn = cheb[ny + N / 2 - n];  // sin(pi n / N)
    const double2 sm = 0.5 * (xa + xb), d = xa - xb;
    x[n * ppc] = sm - sn * d;
    x[(N - n) * ppc] = sm + sn * d;
  }
  __syncthreads();
  lines_dif<NF, 0>(X, tw, nl, ppc, LS);
  for (int w = tid; w < nl * (N / 2 + 1); w += nt) {
    const int l = w % nl, k = w / nl;
    double2* Z = X + (l / ppc) * LS + (l % ppc);
    const int ik = dif_pos<NF>(k) * ppc, in = dif_pos<NF>((N - k) % N) * ppc;
    const double2 zk = Z[ik], zn = Z[in];
    Z[ik] = 0.5 * (zk + zn) + sHalf[l];
    if (k >= 1 && k < N / 2) {
      const double2 dd = zk - zn;
      Z[in] = mk(0.5 * dd.y, -0.5 * dd.x);
    }
  }
  __syncthreads();
  const double s0 = 2.0 / N;
  for (int l = tid; l < nl; l += nt) {
    const int f = l / ppc, pl = l % ppc;
    if (p0 + pl >= P) continue;
    const double2* Z = X + f * LS + pl;
    double2* dst = Rt + (size_t)f * ny * P + pl;
    double2 fo = sF1[l];
    dst[0] = (0.5 * s0) * Z[0];
    dst[P] = s0 * fo;
#pragma unroll 4
    for (int k = 1; k <= N / 2; ++k) {
      dst[(size_t)(2 * k) * P] = (2 * k == N ? 0.5 * s0 : s0) * Z[dif_pos<NF>(k) * ppc];
      if (k < N / 2) {
        fo = fo + Z[dif_pos<NF>(N - k) * ppc];
        dst[(size_t)(2 * k + 1) * P] = s0 * fo;
      }
    }
  }
  __syncthreads();
  for (int w = tid; w < 3 * ny * ppc; w += nt) {
    const int pl = w % ppc, fn = w / ppc;
    if (p0 + pl < P) X[w] = Rt[(size_t)fn * P + pl];
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// stage_pre
//   u = (i kx Dv - i kz g)/k^2, w = (i kz Dv + i kx g)/k^2,
//   omega_x = Dw - i kz v, omega_z = i kx v - Du;  mean mode: u = U, w = W,
//   omega_x = DW, omega_z = -DU.
// Thread (mode, class c, component r) writes component r of u, w, omega_y on
// parity 1-c and of v, omega_x, omega_z on parity c; its derivative chains run
// on component 1-r from n = N down to 0.  All threads then evaluate the six
// Chebyshev series at the nodes: f_j = E_j + O_j, f_{N-j} = E_j - O_j with the
// even/odd partial sums of a_n cos(pi n j / N), for the (N+1)/2 node pairs
// j < N/2.  For even N the middle node needs no products,
// f_{N/2} = sum_m (-1)^m a_{2m}; the thread writing the even coefficients of a
// field sums it on the way, so the node pairs divide evenly over the threads.
// ---------------------------------------------------------------------------
template <typename RN, int MH>
__global__ void __launch_bounds__(128) stage_pre_kernel(Grid g, int B, PencilBufs pb, DevTables t,
                                                        typename cpx<RN>::T* __restrict__ q, int ppc) {
  using CN = typename cpx<RN>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int P = g.P, ny = g.ny, N = g.N;
  // v, omega_y coefficients rounded once to the node precision (every use
  // below is in that precision), then the six fields
  CN* sV = reinterpret_cast<CN*>(smem_raw);  // [ny][ppc]
  CN* sG = sV + ny * ppc;                    // [ny][ppc]
  CN* sC = sG + ny * ppc;                    // [6][ny][ppc]
  const int p0 = blockIdx.x * ppc;
  const int b = blockIdx.y;
  if (pb.active && !pb.active[b]) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  pdl_wait_then_release();  // v, omega_y come from the previous stage
  // FP64 nodes on a grid whose N the FFT plan covers: fast synthesis
  constexpr int NF = 2 * (MH - 1);
  constexpr bool kFastOk = std::is_same<RN, double>::value && ct_plan_ok(NF);
  const bool fast = kFastOk && N == NF;

  for (int w = tid; w < ny * ppc; w += nt) {
    const int pl = w % ppc, n = w / ppc;
    const int p = p0 + pl;
    const size_t o = ((size_t)b * ny + n) * P + p;
    sV[w] = to_node<CN>((p < P) ? pb.V[o] : mk(0.0, 0.0));
    sG[w] = to_node<CN>((p < P) ? pb.G[o] : mk(0.0, 0.0));
  }
  __syncthreads();

  // Recover: the chain of every (mode, class c, component r) is walked by
  // LC = 4 lanes (fixed, so every tile shape sums in the same order).  Lane lc
  // takes a contiguous block of the step pairs (U-step at n_u = nu0 - 2k,
  // V-step at n_u - 1), counted from the top; Dv, D omega_y and then D^2 v are
  // inclusive prefix sums of their terms over k, formed per block and
  // completed by the block totals of the lanes above (shuffles within the
  // 4-lane group); the halvings at n = 0 come last.
  {
    constexpr int LC = 4;
    constexpr int KB = (MH + 1 + LC - 1) / LC;  // step pairs per lane, bound
    const int lc = tid % LC;
    const int chain = tid / LC;  // (mode, combo) as tid did before: pl fastest
    const bool on = chain < 4 * ppc;
    const int pl = chain % ppc;
    const int combo = chain / ppc;
    const int c = combo & 1, r = combo >> 1;
    const int p = p0 + pl;
    const int row = p / g.nxh, ix = p % g.nxh;
    const int fs = 2 * ny * ppc;  // reals per field
    RN* out = reinterpret_cast<RN*>(sC) + 2 * pl + r;
    // middle node f_{N/2} = sum over even n of (-1)^(n/2) a_n, per field
    RN mid[6] = {0, 0, 0, 0, 0, 0};
    auto W = [&](int f, int n, RN x) {
      out[f * fs + n * 2 * ppc] = x;
      if (!fast && (n & 1) == 0) mid[f] = (n & 2) ? mid[f] - x : mid[f] + x;
    };
    // inclusive prefix over the 4-lane group of this lane's block total;
    // returns the exclusive offset
    auto lane_offset = [&](RN tot) {
      RN inc = tot;
#pragma unroll
      for (int o = 1; o < LC; o <<= 1) {
        const RN v = __shfl_up_sync(0xffffffffu, inc, o, LC);
        if (lc >= o) inc = inc + v;
      }
      return inc - tot;
    };
    const bool zero = !on || p >= P || row == g.nz / 2 || (p == 0 && r == 1);
    const bool mean = on && !zero && p == 0;
    if (on && zero) {
      for (int n = lc; n <= N; n += LC) {
        if ((n & 1) == 1 - c) { W(0, n, 0.0); W(2, n, 0.0); W(4, n, 0.0); }
        else { W(1, n, 0.0); W(3, n, 0.0); W(5, n, 0.0); }
      }
    } else if (mean && lc == 0) {
      const double* U = pb.UM + (size_t)b * ny;
      const double* Wm = pb.WM + (size_t)b * ny;
      double du = 0.0, dw = 0.0;
      for (int n = N; n >= 0; --n) {
        if ((n & 1) == 1 - c) {
          W(0, n, U[n]);
          W(2, n, Wm[n]);
          W(4, n, 0.0);
        } else {
          const double un = (n + 1 <= N) ? U[n + 1] : 0.0, wn = (n + 1 <= N) ? Wm[n + 1] : 0.0;
          const double t1 = du + 2.0 * (n + 1) * un, t2 = dw + 2.0 * (n + 1) * wn;
          du = (n == 0) ? 0.5 * t1 : t1;
          dw = (n == 0) ? 0.5 * t2 : t2;
          W(1, n, 0.0);
          W(3, n, dw);
          W(5, n, -du);
        }
      }
    }
    // the scans run on every lane (shuffles); only general modes use them
    const bool gen = on && !zero && !mean;
    const RN kx = gen ? (RN)t.kx[ix] : (RN)0, kz = gen ? (RN)t.kz[row] : (RN)0;
    const RN sg = (r == 0) ? (RN)-1.0 : (RN)1.0;
    const RN ik2 = gen ? sg / (kx * kx + kz * kz) : (RN)0;
    const RN skx = sg * kx, skz = sg * kz;
    const CompT<RN> V{reinterpret_cast<RN*>(sV) + 2 * pl + r, 2 * ppc};
    const CompT<RN> Va{reinterpret_cast<RN*>(sV) + 2 * pl + (1 - r), 2 * ppc};
    const CompT<RN> G{reinterpret_cast<RN*>(sG) + 2 * pl + r, 2 * ppc};
    const CompT<RN> Ga{reinterpret_cast<RN*>(sG) + 2 * pl + (1 - r), 2 * ppc};
    const int nu0 = ((N & 1) == 1 - c) ? N : N + 1;  // first U-step (N + 1: none)
    const int K = nu0 / 2 + 1;                       // step pairs
    const int Bk = (K + LC - 1) / LC;
    const int k0 = lc * Bk;
    RN dvk[KB], dgk[KB], d2k[KB];
    RN sdv = 0, sdg = 0;
#pragma unroll
    for (int j = 0; j < KB; ++j) {
      const int k = k0 + j;
      const int nu = nu0 - 2 * k;
      RN tdv = 0, tdg = 0;
      if (gen && j < Bk && k < K) {
        if (nu + 1 <= N) tdv = (RN)(2 * (nu + 1)) * Va[nu + 1];  // U-step at nu
        if (nu <= N && nu >= 1) tdg = (RN)(2 * nu) * Ga[nu];      // V-step at nu - 1
      }
      sdv = sdv + tdv;
      sdg = sdg + tdg;
      dvk[j] = sdv;
      dgk[j] = sdg;
    }
    const RN odv = lane_offset(sdv), odg = lane_offset(sdg);
    RN sd2 = 0;
#pragma unroll
    for (int j = 0; j < KB; ++j) {
      const int k = k0 + j;
      const int nu = nu0 - 2 * k;
      dvk[j] = dvk[j] + odv;
      dgk[j] = dgk[j] + odg;
      RN td2 = 0;
      if (gen && j < Bk && k < K && nu >= 1) td2 = (RN)(2 * nu) * dvk[j];  // V-step at nu - 1
      sd2 = sd2 + td2;
      d2k[j] = sd2;
    }
    const RN od2 = lane_offset(sd2);
    if (gen) {
#pragma unroll
      for (int j = 0; j < KB; ++j) {
        const int k = k0 + j;
        if (j >= Bk || k >= K) continue;
        const int nu = nu0 - 2 * k, nv = nu - 1;
        if (nu <= N) {
          const RN dv = (nu == 0) ? (RN)0.5 * dvk[j] : dvk[j];
          const RN ga = Ga[nu];
          W(0, nu, ik2 * (kx * dv - kz * ga));  // u
          W(2, nu, ik2 * (kz * dv + kx * ga));  // w
          W(4, nu, G[nu]);                      // omega_y
        }
        if (nv >= 0) {
          const RN h = (nv == 0) ? (RN)0.5 : (RN)1.0;
          const RN d2v = h * (d2k[j] + od2), dg = h * dgk[j];
          const RN va = Va[nv];
          const RN du = ik2 * (kx * d2v - kz * dg);
          const RN dw = ik2 * (kz * d2v + kx * dg);
          W(1, nv, V[nv]);            // v
          W(3, nv, dw - skz * va);    // omega_x = Dw - i kz v
          W(5, nv, skx * va - du);    // omega_z = i kx v - Du
        }
      }
    }
    // middle node: the even coefficients of this chain's fields are spread over
    // its 4 lanes
#pragma unroll
    for (int f = 0; f < 6; ++f)
#pragma unroll
      for (int o = 1; o < LC; o <<= 1) mid[f] = mid[f] + __shfl_xor_sync(0xffffffffu, mid[f], o, LC);
    // this chain wrote the even coefficients of fields 0, 2, 4 (c = 1) or 1, 3, 5 (c = 0)
    if (on && lc == 0 && !fast && (N & 1) == 0 && p < P) {
      RN* qr = reinterpret_cast<RN*>(q);
#pragma unroll
      for (int f = 0; f < 6; ++f)
        if ((f & 1) == 1 - c) qr[2 * (((size_t)(b * 6 + f) * ny + N / 2) * P + p) + r] = mid[f];
    }
  }
  __syncthreads();

  if constexpr (kFastOk) {
    if (fast) {
      const int nl = 6 * ppc;
      const int LS = ny * ppc;
      double2* X = sC;                   // [6][ny][ppc] coefficients, then y, then Z
      double2* sHalf = sC + 6 * ny * ppc;  // [6 ppc] (x_0 + x_N) / 2
      double2* sF1 = sHalf + nl;           // [6 ppc] F_1
      const double* cheb = t.cheb;       // cheb[ny + m] = cos(pi m / N)
      for (int l = tid; l < nl; l += nt) {
        const double2* x = X + (l / ppc) * LS + (l % ppc);
        double2 s1 = mk(0.0, 0.0);
        for (int n = 0; n <= N; ++n) s1 = s1 + cheb[ny + n] * x[n * ppc];
        sF1[l] = s1;
        sHalf[l] = 0.5 * (x[0] + x[N * ppc]);
      }
      __syncthreads();
      for (int w = tid; w < nl * (N / 2); w += nt) {
        const int l = w % nl, n = w / nl;
        double2* x = X + (l / ppc) * LS + (l % ppc);
        if (n == 0) {
          x[0] = sHalf[l];  // y_0; y_{N/2} = x_{N/2} stays
          continue;
        }
        const double2 xa = x[n * ppc], xb = x[(N - n) * ppc];
        const double sn = cheb[ny + N / 2 - n];  // sin(pi n / N)
        const double2 sm = 0.5 * (xa + xb), d = xa - xb;
        x[n * ppc] = sm - sn * d;
        x[(N - n) * ppc] = sm + sn * d;
      }
      __syncthreads();
      lines_dif<NF, 0>(X, t.tw_cheb, nl, ppc, LS);
      // even outputs, and the odd-output differences -i (Z_k - Z_{N-k}) / 2
      // stored in Z_k's own slot (slots of Z_{N-k}, k < N/2, are only read)
      for (int w = tid; w < nl * (NF / 2 + 1); w += nt) {
        const int l = w % nl, k = w / nl;
        const int f = l / ppc, pl = l % ppc, p = p0 + pl;
        double2* Z = X + f * LS + pl;
        const int ik = dif_pos<NF>(k) * ppc;
        const double2 zk = Z[ik];
        const double2 zn = Z[dif_pos<NF>((NF - k) % NF) * ppc];
        if (p < P) q[((size_t)(b * 6 + f) * ny + 2 * k) * P + p] = 0.5 * (zk + zn) + sHalf[l];
        if (k >= 1 && k < NF / 2) {
          const double2 dd = zk - zn;
          Z[ik] = mk(0.5 * dd.y, -0.5 * dd.x);
        }
      }
      __syncthreads();
      // odd outputs: prefix sums from F_1
      for (int l = tid; l < nl; l += nt) {
        const int f = l / ppc, pl = l % ppc, p = p0 + pl;
        if (p >= P) continue;
        const double2* Z = X + f * LS + pl;
        double2* dst = q + ((size_t)(b * 6 + f) * ny) * P + p;
        double2 fo = sF1[l];
        dst[P] = fo;
#pragma unroll 4
        for (int k = 1; k < NF / 2; ++k) {
          fo = fo + Z[dif_pos<NF>(k) * ppc];
          dst[(size_t)(2 * k + 1) * P] = fo;
        }
      }
      return;
    }
  }

  // synthesis of the six fields at the nodes.  Thread (mode pl, group g of
  // nt / ppc) evaluates the node pairs j = g, g + ng, ... of all six fields of
  // its mode: each coefficient it loads feeds all of its outputs, which are
  // independent accumulation chains.
  {
    constexpr int KJ = (MH - 1 + 15) / 16;  // node pairs per thread (ng = nt / ppc >= 16)
    const int ng = nt / ppc;
    const int pl = tid % ppc, gq = tid / ppc;
    const int J = (N + 1) / 2;  // node pairs (j, N - j), j < N/2
    const RN* cheb = cheb_table<RN>(t);
    if (gq < ng) {
      CN E[6][KJ], O[6][KJ];
#pragma unroll
      for (int f = 0; f < 6; ++f)
#pragma unroll
        for (int k = 0; k < KJ; ++k) {
          E[f][k] = czero<CN>();
          O[f][k] = czero<CN>();
        }
      const CN* col = sC + pl;
      // even and odd n in one iteration, so that neither update is predicated
      auto accumulate = [&](int n, CN (&acc)[6][KJ]) {
        CN cf[6];
#pragma unroll
        for (int f = 0; f < 6; ++f) cf[f] = col[((size_t)f * ny + n) * ppc];
#pragma unroll
        for (int k = 0; k < KJ; ++k) {
          const int j = gq + ng * k;
          const RN c = cheb[(size_t)min(j, N) * ny + n];
#pragma unroll
          for (int f = 0; f < 6; ++f) acc[f][k] = acc[f][k] + c * cf[f];
        }
      };
      for (int n = 0; n + 1 <= N; n += 2) {
        accumulate(n, E);
        accumulate(n + 1, O);
      }
      if ((N & 1) == 0) accumulate(N, E);
      const int p = p0 + pl;
      if (p < P) {
#pragma unroll
        for (int k = 0; k < KJ; ++k) {
          const int j = gq + ng * k;
          if (j >= J) continue;
#pragma unroll
          for (int f = 0; f < 6; ++f) {
            CN* dst = q + ((size_t)(b * 6 + f) * ny) * P + p;
            dst[(size_t)j * P] = E[f][k] + O[f][k];
            dst[(size_t)(N - j) * P] = E[f][k] - O[f][k];
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// stage_post
// Analysis: a_n = 2/(N cb_n) sum_j f_j cos(pi n j / N) / cb_j (cb_0 = cb_N = 2),
// node pairs (j, N-j) folded by the parity of n.
// Implicit part, with c = alpha/beta and the shifted unknowns
// g' = g^k + c g^{k-1}, phi' = phi^k + c phi^{k-1}, v' = v^k + c v^{k-1}:
//   (D^2 - lam) g'   = -((1 + c) g + dt (gamma h_g + zeta h_g')) / (beta dt nu)
//   (D^2 - lam) phi' = -((1 + c) phi + dt (gamma h_v + zeta h_v')) / (beta dt nu),
//   (D^2 - k^2) v'   = phi',   phi = (D^2 - k^2) v^{k-1},
// lam = k^2 + 1/(beta dt nu).  (D^2 - k^2) X = (D^2 - lam) X + X/(beta dt nu)
// holds for every coefficient row, so this is the same tau discretisation as
// the plain form without derivatives of the old fields.  The solve is linear
// in its right-hand side, so the factor -1/(beta dt nu), the same for every
// coefficient of a stage, is folded into the elimination factors e of the
// Helmholtz tables on the host: the kernels form (1 + c) g + dt (...) only.
// The wall rows of g' and v' carry c times the old wall values; the influence
// matrix fixes Dv'(+-1) = c Dv^{k-1}(+-1).  Then g^k = g' - c g^{k-1},
// v^k = v' - c v^{k-1}.
//   h_g = i kz H_x - i kx H_z,  h_v = -k^2 H_y - D(i kx H_x + i kz H_z).
// Thread (mode, class c, component r, equation e): e = 0 omega_y on parity
// 1-c, e = 1 v on parity c.  The mean mode solves U at constant flow rate
// (e = 0) and W (e = 1) on parity c, real component only.
// ---------------------------------------------------------------------------
// Lanes per system of the per-tile form: four under the no-slip top (the
// scan solves of stage_scan.cuh), one under the free-slip top.
template <int TOP>
constexpr int post_tile_lanes() { return TOP == 0 ? 4 : 1; }

template <typename RN, int MH, int TOP>
__global__ void __launch_bounds__(64 * post_tile_lanes<TOP>()) stage_post_kernel(Grid g, int B, PencilBufs pb, DevTables t,
                                                        const typename cpx<RN>::T* __restrict__ hn, StageCoef sc,
                                                        int ppc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int P = g.P, ny = g.ny, N = g.N;
  const int Mh = t.tau.Mh;
  using CN = typename cpx<RN>::T;
  double2* sH = reinterpret_cast<double2*>(smem_raw);  // [3][ny][ppc] nodes, then coefficients (RN)
  double2* sV = sH + 3 * ny * ppc;                      // [ny][ppc]
  double2* sG = sV + ny * ppc;
  // previous right-hand sides h_v', h_g' in the node precision (FP64-sized slots)
  CN* sHV = reinterpret_cast<CN*>(sG + ny * ppc);
  CN* sHG = reinterpret_cast<CN*>(sG + 2 * ny * ppc);
  double* sh = reinterpret_cast<double*>(sG + 3 * ny * ppc);  // helm [2][4][Mh][ppc] of this stage
  double* sp = sh + 2 * 4 * Mh * ppc;                        // pois [2][4][Mh][ppc]
  double* svh = sp + 2 * 4 * Mh * ppc;                       // vh [2][Mh][ppc]
  double* ss = svh + 2 * Mh * ppc;                           // helm_isq, pois_isq, vh_idv [3][2][ppc]
  const int p0 = blockIdx.x * ppc;
  const int b = blockIdx.y;
  if (pb.active && !pb.active[b]) return;
  const int tid = threadIdx.x, nt = blockDim.x;

  // ---- load the tile (asynchronous copies, all in flight before the wait)
  for (int w = tid; w < ny * ppc; w += nt) {
    const int pl = w % ppc, n = w / ppc;
    const int p = min(p0 + pl, P - 1);
    const size_t o = ((size_t)b * ny + n) * P + p;
    cp_async_elem(sV + w, pb.V + o);
    cp_async_elem(sG + w, pb.G + o);
    cp_async_elem(sHV + w, reinterpret_cast<const CN*>(pb.HVP) + o);
    cp_async_elem(sHG + w, reinterpret_cast<const CN*>(pb.HGP) + o);
  }
  for (int w = tid; w < 2 * 4 * Mh * ppc; w += nt) {
    const int pl = w % ppc, qq = w / ppc;  // qq = (sig * 4 + f) * Mh + i
    const int p = min(p0 + pl, P - 1);
    cp_async_elem(sh + w, t.tau.helm + ((size_t)sc.k * 2 * 4 * Mh + qq) * P + p);
    cp_async_elem(sp + w, t.tau.pois + (size_t)qq * P + p);
  }
  for (int w = tid; w < 2 * Mh * ppc; w += nt) {
    const int pl = w % ppc, qq = w / ppc;
    const int p = min(p0 + pl, P - 1);
    cp_async_elem(svh + w, t.tau.vh + ((size_t)sc.k * 2 * Mh + qq) * P + p);
  }
  for (int w = tid; w < 2 * ppc; w += nt) {
    const int pl = w % ppc, sig = w / ppc;
    const int p = min(p0 + pl, P - 1);
    cp_async_elem(ss + (0 * 2 + sig) * ppc + pl, t.tau.helm_isq + (size_t)(sc.k * 2 + sig) * P + p);
    cp_async_elem(ss + (1 * 2 + sig) * ppc + pl, t.tau.pois_isq + (size_t)sig * P + p);
    cp_async_elem(ss + (2 * 2 + sig) * ppc + pl, t.tau.vh_idv + (size_t)(sc.k * 2 + sig) * P + p);
  }
  // everything above is independent of the nonlinear term; H comes from the
  // preceding kernel
  pdl_wait_then_release();
  // nodal values in the node precision, in the first bytes of the sH region
  CN* sN = reinterpret_cast<CN*>(sH);
  for (int w = tid; w < 3 * ny * ppc; w += nt) {
    const int pl = w % ppc, fn = w / ppc;  // fn = f * ny + n
    const int p = min(p0 + pl, P - 1);
    cp_async_elem(sN + w, hn + ((size_t)b * 3 * ny + fn) * P + p);
  }
  cp_async_wait_all();
  __syncthreads();

  // ---- Chebyshev analysis of H_x, H_y, H_z (in place after a barrier)
  constexpr int NF = 2 * (MH - 1);
  bool analysed = false;
  if constexpr (std::is_same<RN, double>::value && ct_plan_ok(NF)) {
    if (N == NF) {
      analysis_fft<NF>(sH, ppc, ny, P, p0, reinterpret_cast<double2*>(ss + 6 * ppc), t.cheb, t.tw_cheb,
                       pb.R + (size_t)b * 3 * ny * P + p0);
      analysed = true;
    }
  }
  if (!analysed) {
    // Thread (mode pl, group g of GA) computes the coefficients n = g, g+GA, ...
    // of the three fields of its mode: every pair f_j, f_{N-j} it loads feeds
    // all of its outputs, and the outputs are independent accumulation chains.
    // n and g share their parity, so the folding sign is fixed per thread.
    constexpr int GA = 8 * post_tile_lanes<TOP>();
    constexpr int KN = (2 * MH + GA - 1) / GA;  // n values per thread
    const int pl = tid % ppc, gq = tid / ppc;  // blockDim = GA ppc
    const RN* cheb = cheb_table<RN>(t);
    const RN sg = (gq & 1) ? (RN)-1.0 : (RN)1.0;
    CN a[3][KN];
    const CN* colf[3];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      colf[f] = sN + (size_t)f * ny * ppc + pl;
      const CN w0 = (RN)0.5 * (colf[f][0] + sg * colf[f][N * ppc]);  // j = 0 and j = N weigh 1/2
#pragma unroll
      for (int k = 0; k < KN; ++k) a[f][k] = w0;
    }
    for (int j = 1; 2 * j < N; ++j) {
      CN fold[3];
#pragma unroll
      for (int f = 0; f < 3; ++f) fold[f] = colf[f][j * ppc] + sg * colf[f][(N - j) * ppc];
#pragma unroll
      for (int k = 0; k < KN; ++k) {
        const int n = gq + GA * k;
        const RN c = cheb[(size_t)min(n, N) * ny + j];
#pragma unroll
        for (int f = 0; f < 3; ++f) a[f][k] = a[f][k] + c * fold[f];
      }
    }
    CN acc[3][KN];
    const RN s0 = (RN)2.0 / (RN)N;
#pragma unroll
    for (int k = 0; k < KN; ++k) {
      const int n = gq + GA * k;
      const RN cbn = (n == 0 || n == N) ? (RN)2.0 : (RN)1.0;
      const RN cH = ((N & 1) == 0) ? cheb[(size_t)min(n, N) * ny + N / 2] : (RN)0.0;
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        CN v = a[f][k];
        if ((N & 1) == 0) v = v + cH * colf[f][(N / 2) * ppc];
        acc[f][k] = (s0 / cbn) * v;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KN; ++k) {
      const int n = gq + GA * k;
      if (n <= N) {
#pragma unroll
        for (int f = 0; f < 3; ++f) sN[((size_t)f * ny + n) * ppc + pl] = acc[f][k];
      }
    }
    __syncthreads();
  }

  if constexpr (TOP == 0) {
    // ---- implicit solves, system (mode pl, class c, component r, equation
    // e) on the four lanes q of a group
    const int q = tid & 3, sys = tid >> 2;
    const int pl = sys % ppc;
    const int combo = sys / ppc;
    const int p = p0 + pl;
    const int c = combo & 1, r = (combo >> 1) & 1, e = combo >> 2;
    const int row = p / g.nxh, ix = p % g.nxh;
    // a whole group is live or idle together
    if (p < P && row != g.nz / 2 && (p != 0 || r == 0)) {
      const double cc = sc.alpha / sc.beta;
      const double* rowc = t.tau.rowc;
      const CN* Hx = reinterpret_cast<const CN*>(sH) + pl;
      const CN* Hy = Hx + ny * ppc;
      const CN* Hz = Hy + ny * ppc;
      auto helm = [&](int sig) { return TabSm{sh + sig * 4 * Mh * ppc + pl, Mh, ppc}; };
      auto comp = [](auto z, int qd) { return qd == 0 ? z.x : z.y; };
      if (p == 0) {
        mean_scan<MH, RN>(N, ny, ppc, c, e, (e == 0 ? pb.UM : pb.WM) + (size_t)b * ny,
                          (e == 0 ? pb.HXP : pb.HZP) + (size_t)b * ny, (e == 0) ? Hx : Hz, cc, sc, helm(c),
                          ss[(0 * 2 + c) * ppc + pl], rowc, t.tau.u1 + (size_t)sc.k * Mh, t.tau.u1_iflux[sc.k], q);
      } else {
        const double kx = t.kx[ix], kz = t.kz[row], k2 = kx * kx + kz * kz;
        const double sgn = (r == 0) ? -1.0 : 1.0;
        if (e == 0) {
          // wall-normal vorticity, parity 1 - c
          const int sq = 1 - c;
          const CompS Gc{reinterpret_cast<double*>(sG) + 2 * pl + r, 2 * ppc};
          const CompT<RN> HGc{reinterpret_cast<RN*>(sHG) + 2 * pl + r, 2 * ppc};
          omega_scan<MH, RN>(N, ny, ppc, sq, Gc, HGc, Hx, Hz, r, sgn, kx, kz, cc, sc, helm(sq),
                             ss[(0 * 2 + sq) * ppc + pl], rowc, q);
        } else {
          // wall-normal velocity, parity c
          const int sv = c;
          const CompS Vc{reinterpret_cast<double*>(sV) + 2 * pl + r, 2 * ppc};
          const CompT<RN> HVc{reinterpret_cast<RN*>(sHV) + 2 * pl + r, 2 * ppc};
          const size_t vo = (size_t)b * P + p;
          const double vw =
              fma_rn(sc.theta, comp(pb.vw_new[vo], r) - comp(pb.vw_old[vo], r), comp(pb.vw_old[vo], r));
          const TabSm TP{sp + sv * 4 * Mh * ppc + pl, Mh, ppc};
          v_scan<MH, RN>(N, ny, ppc, sv, Vc, HVc, Hx, Hy, Hz, r, sgn, kx, kz, k2, cc, sc, helm(sv),
                         ss[(0 * 2 + sv) * ppc + pl], TP, ss[(1 * 2 + sv) * ppc + pl], svh + sv * Mh * ppc + pl,
                         ppc, ss[(2 * 2 + sv) * ppc + pl], vw, rowc, q);
        }
      }
    }
  } else {
    // ---- implicit solves under a free-slip top: each thread forms the
    // affine family of its parity and publishes its sums; the closure follows
    // the barrier.  Thread (mode, class c, component r, equation e) as above;
    // its partner of the other parity is class 1 - c.
    double* xch = reinterpret_cast<double*>(ss + 6 * ppc) + 12 * ppc;  // [8 ppc threads][6]
    const int pl = tid % ppc;
    const int combo = tid / ppc;
    const int p = p0 + pl;
    const int c = combo & 1, r = (combo >> 1) & 1, e = combo >> 2;
    const int row = p / g.nxh, ix = p % g.nxh;
    const bool live = p < P && combo < 8 && row != g.nz / 2 && !(p == 0 && r == 1);
    const double cc = sc.alpha / sc.beta;
    const double* rowc = t.tau.rowc;
    const CN* Hx = reinterpret_cast<const CN*>(sH) + pl;
    const CN* Hy = Hx + ny * ppc;
    const CN* Hz = Hy + ny * ppc;
    auto helm = [&](int sig) { return TabSm{sh + sig * 4 * Mh * ppc + pl, Mh, ppc}; };
    auto comp = [](auto z, int qd) { return qd == 0 ? z.x : z.y; };
    const int pc = min(p, P - 1);
    // table sums of both parities: sum Q, sum n^2 Q of this stage; A, B of vh
    auto qs = [&](int sig, int w) { return t.tau.helm_top[((size_t)(sc.k * 2 + sig) * 2 + w) * P + pc]; };
    auto vs = [&](int sig, int w) { return t.tau.vh_top[((size_t)(sc.k * 2 + sig) * 2 + w) * P + pc]; };
    double* mine = xch + tid * 6;
    const double* other = xch + ((combo ^ 1) * ppc + pl) * 6;
    RegArr<MH> f;
    int sig = 0;
    if (live) {
      if (p == 0) {
        // mean mode: U (e = 0) at constant flow rate, W (e = 1), parity c
        sig = c;
        mean_open_affine<MH, RN>(f, N, ny, ppc, sig, (e == 0 ? pb.UM : pb.WM) + (size_t)b * ny,
                                 (e == 0 ? pb.HXP : pb.HZP) + (size_t)b * ny, (e == 0) ? Hx : Hz, cc, sc, helm(sig),
                                 rowc, mine);
      } else if (e == 0) {
        // wall-normal vorticity, parity 1 - c
        sig = 1 - c;
        const CompS Gc{reinterpret_cast<double*>(sG) + 2 * pl + r, 2 * ppc};
        const CompT<RN> HGc{reinterpret_cast<RN*>(sHG) + 2 * pl + r, 2 * ppc};
        omega_open_affine<MH, RN>(f, N, ny, ppc, sig, Gc, HGc, HGc, Hx, Hz, r, (r == 0) ? -1.0 : 1.0, t.kx[ix],
                                  t.kz[row], cc, sc, helm(sig), rowc, mine);
      } else {
        // wall-normal velocity, parity c: phi_p and v_p as in the no-slip
        // channel (Dirichlet rows of both), then the sums of the free-slip rows
        sig = c;
        const double kx = t.kx[ix], kz = t.kz[row], k2 = kx * kx + kz * kz;
        const CompS Vc{reinterpret_cast<double*>(sV) + 2 * pl + r, 2 * ppc};
        const CompT<RN> HVc{reinterpret_cast<RN*>(sHV) + 2 * pl + r, 2 * ppc};
        const size_t vo = (size_t)b * P + p;
        const double vw =
            fma_rn(sc.theta, comp(pb.vw_new[vo], r) - comp(pb.vw_old[vo], r), comp(pb.vw_old[vo], r));
        const TabSm TP{sp + sig * 4 * Mh * ppc + pl, Mh, ppc};
        v_open_part<MH, RN>(f, N, ny, ppc, sig, Vc, HVc, HVc, Hx, Hy, Hz, r, (r == 0) ? -1.0 : 1.0, kx, kz, k2, cc,
                            sc, helm(sig), ss[(0 * 2 + sig) * ppc + pl], TP, ss[(1 * 2 + sig) * ppc + pl], vw, rowc,
                            mine);
      }
    }
    __syncthreads();
    if (live) {
      const double* se = sig == 0 ? mine : other;
      const double* so = sig == 0 ? other : mine;
      const int M = (N - sig) / 2 + 1;
      if (p == 0) {
        double* X = (e == 0 ? pb.UM : pb.WM) + (size_t)b * ny;
        double xe, xo, fc = 0.0;
        if (e == 1) {
          close_neumann_top(se, so, qs(0, 0), qs(1, 0), qs(0, 1), qs(1, 1), cc, &xe, &xo);
        } else {
          // forcing response (even parity) and int Q_e
          const double* u1 = t.tau.u1 + (size_t)sc.k * Mh;
          const TabSm He = helm(0);
          double us = 0.0, u2 = 0.0, uw = 0.0, wq = 0.0;
          for (int i = 0; i < N / 2 + 1; ++i) {
            const double n = 2 * i, w = 2.0 / (1.0 - n * n);
            us += u1[i];
            u2 = fma_rn(n * n, u1[i], u2);
            uw = fma_rn(w, u1[i], uw);
            wq = fma_rn(w, i == 0 ? 1.0 : He.Q(i), wq);
          }
          close_free_slip_mean(se, so, qs(0, 0), qs(1, 0), qs(0, 1), qs(1, 1), wq, us, u2, uw, cc, sc.flux, &xe,
                               &xo, &fc);
        }
        tau_close<MH>(N, sig, f, helm(sig), sig == 0 ? xe : xo);
#pragma unroll
        for (int i = 0; i < MH; ++i)
          if (i < M) {
            const int n = 2 * i + sig;
            double v = fma_rn(-cc, X[n], f[i]);
            if (e == 0 && sig == 0) v = fma_rn(fc, t.tau.u1[(size_t)sc.k * Mh + i], v);
            X[n] = v;
          }
      } else if (e == 0) {
        const CompS Gc{reinterpret_cast<double*>(sG) + 2 * pl + r, 2 * ppc};
        double xe, xo;
        close_neumann_top(se, so, qs(0, 0), qs(1, 0), qs(0, 1), qs(1, 1), cc, &xe, &xo);
        tau_close<MH>(N, sig, f, helm(sig), sig == 0 ? xe : xo);
#pragma unroll
        for (int i = 0; i < MH; ++i)
          if (i < M) {
            const int n = 2 * i + sig;
            Gc[n] = fma_rn(-cc, Gc[n], f[i]);
          }
      } else {
        const CompS Vc{reinterpret_cast<double*>(sV) + 2 * pl + r, 2 * ppc};
        double ce, co;
        close_free_slip_v(se, so, vs(0, 0), vs(1, 0), vs(0, 1), vs(1, 1), cc, &ce, &co);
        const double cI = sig == 0 ? ce : co;
        const double* vh = svh + sig * Mh * ppc + pl;
#pragma unroll
        for (int i = 0; i < MH; ++i)
          if (i < M) {
            const int n = 2 * i + sig;
            Vc[n] = fma_rn(-cc, Vc[n], fma_rn(cI, vh[i * ppc], f[i]));
          }
      }
    }
  }
  __syncthreads();

  // ---- store the tile
  for (int w = tid; w < ny * ppc; w += nt) {
    const int pl2 = w % ppc, n = w / ppc;
    const int p2 = p0 + pl2;
    if (p2 >= P) continue;
    const size_t o = ((size_t)b * ny + n) * P + p2;
    pb.V[o] = sV[w];
    pb.G[o] = sG[w];
    reinterpret_cast<CN*>(pb.HVP)[o] = sHV[w];
    reinterpret_cast<CN*>(pb.HGP)[o] = sHG[w];
  }
}

// ---------------------------------------------------------------------------
// stage_post, batched form.  The same arithmetic as stage_post_kernel, mapped
// for many modes: one thread per (mode, class c, component r) solves both
// equations of its class (omega_y on parity 1-c, then v on parity c), so every
// warp carries the same FP64 work, and only the Chebyshev coefficients of H
// are staged in shared memory (3 ny complex per mode, against 7 ny complex
// plus the tau tables in the per-tile form), which lets four times as many
// modes be resident per SM.  The state, the previous right-hand sides and the
// tau tables are read and written in place in global memory by the thread
// that owns them; lanes (mode, r) make these accesses contiguous.  The
// analysis runs field by field with four threads per mode (n = q + 4k); each
// coefficient is accumulated in the same order as in the per-tile form.
// ---------------------------------------------------------------------------
// Five CTAs per SM with up to 65 nodes: the register budget (168) holds the
// solves' one array of coefficients, and the shared tile (41.6 KB at 65
// nodes in FP32, 44.6 KB with the free-slip exchange slots) allows five.
template <int MH, int TOP>
constexpr int post_batched_min_ctas() { return MH <= 33 ? 5 : 1; }

template <typename RN, int MH, int TOP>
__global__ void __launch_bounds__(64, post_batched_min_ctas<MH, TOP>()) stage_post_batched_kernel(Grid g, int B, PencilBufs pb, DevTables t,
                                                                const typename cpx<RN>::T* __restrict__ hn,
                                                                StageCoef sc, int ppc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using CN = typename cpx<RN>::T;
  const int P = g.P, ny = g.ny, N = g.N;
  const int Mh = t.tau.Mh;
  double2* sH = reinterpret_cast<double2*>(smem_raw);  // [3][ny][ppc] coefficients
  CN* sN = reinterpret_cast<CN*>(smem_raw);             // [3][ny][ppc] nodal values, same bytes
  const int p0 = blockIdx.x * ppc;
  const int b = blockIdx.y;
  if (pb.active && !pb.active[b]) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  // FP32 nodes: the previous right-hand sides (FP32 pairs) are staged in shared
  // memory behind the node tile, issued before the wait for H; the new ones go
  // straight to global memory.  Both tiles arrive by asynchronous copies.
  constexpr bool kStageHV = sizeof(RN) == 4 && kPostStageHV, kStageHG = sizeof(RN) == 4 && kPostStageHG;
  CN* sHVt = sN + 3 * ny * ppc;
  CN* sHGt = sHVt + (kStageHV ? ny * ppc : 0);
  if (kStageHV || kStageHG) {
    for (int w = tid; w < ny * ppc; w += nt) {
      const int pl = w % ppc, n = w / ppc;
      const size_t o = ((size_t)b * ny + n) * P + min(p0 + pl, P - 1);
      if (kStageHV) cp_async_elem(sHVt + w, reinterpret_cast<const CN*>(pb.HVP) + o);
      if (kStageHG) cp_async_elem(sHGt + w, reinterpret_cast<const CN*>(pb.HGP) + o);
    }
  }
  pdl_wait_then_release();  // H comes from the preceding kernel
  for (int w = tid; w < 3 * ny * ppc; w += nt) {
    const int pl = w % ppc, fn = w / ppc;  // fn = f * ny + n
    const int p = min(p0 + pl, P - 1);
    cp_async_elem(sN + w, hn + ((size_t)b * 3 * ny + fn) * P + p);
  }
  cp_async_wait_all();
  __syncthreads();
  // thread (mode pl, class c, component r).  Under the no-slip top each warp
  // holds one class (16 or more modes per CTA); under the free-slip top the
  // two classes of a (mode, component) are neighbouring lanes, whose parity
  // closures exchange their sums by shuffles.
  const int r = TOP ? (tid >> 1) & 1 : tid & 1;
  const int pl = TOP ? tid >> 2 : (tid >> 1) % ppc;
  const int c = TOP ? tid & 1 : tid / (2 * ppc);

  // ---- Chebyshev analysis of H_z, H_y, H_x, coefficients in the node
  // precision over the nodal values of the same field (a barrier between
  // reading and writing each field).
  constexpr int NF = 2 * (MH - 1);
  bool analysed = false;
  if constexpr (std::is_same<RN, double>::value && ct_plan_ok(NF)) {
    if (N == NF) {
      analysis_fft<NF>(sH, ppc, ny, P, p0, sH + 3 * ny * ppc, t.cheb, t.tw_cheb,
                       pb.R + (size_t)b * 3 * ny * P + p0);
      analysed = true;
    }
  }
  if (!analysed) {
    constexpr int KN = (2 * MH + 3) / 4;  // n values per thread
    const int qd = r + 2 * c;             // n = qd + 4k, parity of n = r
    const RN* cheb = cheb_table<RN>(t);
    const RN sg = r ? (RN)-1.0 : (RN)1.0;
    for (int f = 2; f >= 0; --f) {
      CN acc[KN];
      analysis_sums<RN, KN>(sN + (size_t)f * ny * ppc + pl, ppc, N, ny, cheb, qd, 4, sg, acc);
      __syncthreads();
#pragma unroll
      for (int k = 0; k < KN; ++k) {
        const int n = qd + 4 * k;
        if (n <= N) sN[((size_t)f * ny + n) * ppc + pl] = acc[k];
      }
    }
    __syncthreads();
  }

  if constexpr (TOP == 0) {
    // ---- implicit solves (no barrier below)
    const int p = p0 + pl;
    if (p >= P) return;
    if (p / g.nxh == g.nz / 2) return;  // Nyquist row stays zero
    const CN* Hx = sN + pl;
    const CN* Hy = Hx + ny * ppc;
    const CN* Hz = Hy + ny * ppc;
    const size_t base = 2 * ((size_t)b * ny * P + p) + r;  // component r of element n at base + 2 P n
    const CompT<RN> HGr = kStageHG ? CompT<RN>{reinterpret_cast<RN*>(sHGt) + 2 * pl + r, 2 * ppc}
                                   : CompT<RN>{reinterpret_cast<RN*>(pb.HGP) + base, 2 * P};
    const CompT<RN> HVr = kStageHV ? CompT<RN>{reinterpret_cast<RN*>(sHVt) + 2 * pl + r, 2 * ppc}
                                   : CompT<RN>{reinterpret_cast<RN*>(pb.HVP) + base, 2 * P};
    // The class c is uniform over each warp for tiles of 16 or more modes, so
    // for up to 65 nodes (MH <= 33) the solve is compiled once per class: every
    // parity-dependent factor (2 (n + 1), n^2, the row bounds) becomes a
    // constant.  Larger buckets keep one run-time class (their unrolled code
    // would double).  The arithmetic is the same either way: the factors are
    // exact small integers and every fused operation is pinned.
    auto solve = [&](auto cls) {
      post_solve_noslip<MH, RN, false>(nullptr, 0, cls, g, pb, t, sc, b, p, r, Hx, Hy, Hz, ppc, HGr, HVr);
    };
    if constexpr (MH <= 33) {
      if (c == 0) solve(std::integral_constant<int, 0>{});
      else solve(std::integral_constant<int, 1>{});
    } else {
      solve(c);
    }
  } else {
    // ---- implicit solves under a free-slip top, in two closures (omega_y or
    // the mean flow, then v), each closed by the pair of class threads
    // (c, 1 - c) of a (mode, component), neighbouring lanes that exchange
    // their sums by shuffles; every lane of the warp takes part in both
    // exchanges
    const int p = p0 + pl;
    const int pc = min(p, P - 1);
    const int row = pc / g.nxh, ix = pc % g.nxh;
    const bool live = p < P && row != g.nz / 2;
    const bool mean = p == 0;
    const double cc = sc.alpha / sc.beta;
    const double* rowc = t.tau.rowc;
    const CN* Hx = sN + pl;
    const CN* Hy = Hx + ny * ppc;
    const CN* Hz = Hy + ny * ppc;
    auto comp = [](auto z, int qq) { return qq == 0 ? z.x : z.y; };
    auto helm = [&](int sig) { return TabSm{t.tau.helm + (size_t)(sc.k * 2 + sig) * 4 * Mh * P + pc, Mh, P}; };
    auto helm_isq = [&](int sig) { return t.tau.helm_isq[(size_t)(sc.k * 2 + sig) * P + pc]; };
    auto qs = [&](int sig, int w) { return t.tau.helm_top[((size_t)(sc.k * 2 + sig) * 2 + w) * P + pc]; };
    auto vs = [&](int sig, int w) { return t.tau.vh_top[((size_t)(sc.k * 2 + sig) * 2 + w) * P + pc]; };
    const size_t base = 2 * ((size_t)b * ny * P + pc) + r;  // component r of element n at base + 2 P n
    const double sgn = (r == 0) ? -1.0 : 1.0;
    RegArr<MH> f;
    // first closure: the mean mode (U for r = 0, W for r = 1) on parity c, or
    // omega_y on parity 1 - c
    {
      const int sig = mean ? c : 1 - c;
      const int M = (N - sig) / 2 + 1;
      double mine[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      if (live) {
        if (mean) {
          mean_open_affine<MH, RN>(f, N, ny, ppc, sig, (r == 0 ? pb.UM : pb.WM) + (size_t)b * ny,
                                   (r == 0 ? pb.HXP : pb.HZP) + (size_t)b * ny, (r == 0) ? Hx : Hz, cc, sc, helm(sig),
                                   rowc, mine);
        } else {
          const CompS Gc{reinterpret_cast<double*>(pb.G) + base, 2 * P};
          const CompT<RN> HGc{reinterpret_cast<RN*>(pb.HGP) + base, 2 * P};
          const CompT<RN> HGr = kStageHG ? CompT<RN>{reinterpret_cast<RN*>(sHGt) + 2 * pl + r, 2 * ppc} : HGc;
          omega_open_affine<MH, RN>(f, N, ny, ppc, sig, Gc, HGr, HGc, Hx, Hz, r, sgn, t.kx[ix], t.kz[row], cc, sc,
                                    helm(sig), rowc, mine);
        }
      }
      // the mate (other class, same mode and component) is the neighbouring lane
      double se[6], so[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const double other = __shfl_xor_sync(0xffffffffu, mine[k], 1);
        se[k] = sig == 0 ? mine[k] : other;
        so[k] = sig == 0 ? other : mine[k];
      }
      if (live) {
        double xe, xo, fc = 0.0;
        if (mean && r == 0) {
          const double* u1 = t.tau.u1 + (size_t)sc.k * Mh;
          const TabSm He = helm(0);
          double us = 0.0, u2 = 0.0, uw = 0.0, wq = 0.0;
          for (int i = 0; i < N / 2 + 1; ++i) {
            const double n = 2 * i, w = 2.0 / (1.0 - n * n);
            us += u1[i];
            u2 = fma_rn(n * n, u1[i], u2);
            uw = fma_rn(w, u1[i], uw);
            wq = fma_rn(w, i == 0 ? 1.0 : He.Q(i), wq);
          }
          close_free_slip_mean(se, so, qs(0, 0), qs(1, 0), qs(0, 1), qs(1, 1), wq, us, u2, uw, cc, sc.flux, &xe,
                               &xo, &fc);
        } else {
          close_neumann_top(se, so, qs(0, 0), qs(1, 0), qs(0, 1), qs(1, 1), cc, &xe, &xo);
        }
        tau_close<MH>(N, sig, f, helm(sig), sig == 0 ? xe : xo);
        if (mean) {
          double* X = (r == 0 ? pb.UM : pb.WM) + (size_t)b * ny;
#pragma unroll
          for (int i = 0; i < MH; ++i)
            if (i < M) {
              const int n = 2 * i + sig;
              double v = fma_rn(-cc, X[n], f[i]);
              if (r == 0 && sig == 0) v = fma_rn(fc, t.tau.u1[(size_t)sc.k * Mh + i], v);
              X[n] = v;
            }
        } else {
          const CompS Gc{reinterpret_cast<double*>(pb.G) + base, 2 * P};
#pragma unroll
          for (int i = 0; i < MH; ++i)
            if (i < M) {
              const int n = 2 * i + sig;
              Gc[n] = fma_rn(-cc, Gc[n], f[i]);
            }
        }
      }
    }
    // second closure: v on parity c (every mode but the mean)
    {
      const int sig = c;
      const int M = (N - sig) / 2 + 1;
      double mine[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      const bool on = live && !mean;
      const CompS Vc{reinterpret_cast<double*>(pb.V) + base, 2 * P};
      if (on) {
        const double kx = t.kx[ix], kz = t.kz[row], k2 = kx * kx + kz * kz;
        const CompT<RN> HVc{reinterpret_cast<RN*>(pb.HVP) + base, 2 * P};
        const CompT<RN> HVr = kStageHV ? CompT<RN>{reinterpret_cast<RN*>(sHVt) + 2 * pl + r, 2 * ppc} : HVc;
        const size_t vo = (size_t)b * P + pc;
        const double vw =
            fma_rn(sc.theta, comp(pb.vw_new[vo], r) - comp(pb.vw_old[vo], r), comp(pb.vw_old[vo], r));
        const TabSm TP{t.tau.pois + (size_t)sig * 4 * Mh * P + pc, Mh, P};
        v_open_part<MH, RN>(f, N, ny, ppc, sig, Vc, HVr, HVc, Hx, Hy, Hz, r, sgn, kx, kz, k2, cc, sc, helm(sig),
                            helm_isq(sig), TP, t.tau.pois_isq[(size_t)sig * P + pc], vw, rowc, mine);
      }
      double se[6], so[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const double other = __shfl_xor_sync(0xffffffffu, mine[k], 1);
        se[k] = sig == 0 ? mine[k] : other;
        so[k] = sig == 0 ? other : mine[k];
      }
      if (on) {
        double ce, co;
        close_free_slip_v(se, so, vs(0, 0), vs(1, 0), vs(0, 1), vs(1, 1), cc, &ce, &co);
        const double cI = sig == 0 ? ce : co;
        const double* vh = t.tau.vh + (size_t)(sc.k * 2 + sig) * Mh * P + pc;
#pragma unroll
        for (int i = 0; i < MH; ++i)
          if (i < M) {
            const int n = 2 * i + sig;
            Vc[n] = fma_rn(-cc, Vc[n], fma_rn(cI, vh[(size_t)i * P], f[i]));
          }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// The implicit half for more than 65 nodes (no-slip top), in two launches.
// One parity of one unknown then holds up to 101 coefficients, more than a
// thread's registers next to the rest of the solve, and the node tile of H
// (3 ny ppc values) would leave one or two CTAs per SM.  So:
//   stage_post_analysis_kernel: the Chebyshev analysis of H, a tile of modes
//     at a time, written over the nodal values in place (a CTA reads all the
//     nodes of its modes before it writes their coefficients);
//   stage_post_wide_kernel: one thread per (mode, class, component) as in the
//     batched form, reading the coefficients of H from global memory and
//     keeping its array of coefficients in a column of shared memory.
// The per-output arithmetic of both halves is that of the batched form.
// ---------------------------------------------------------------------------
template <typename RN, int MH>
__global__ void __launch_bounds__(256) stage_post_analysis_kernel(Grid g, int B, PencilBufs pb, DevTables t,
                                                                  typename cpx<RN>::T* __restrict__ hn, int ppc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using CN = typename cpx<RN>::T;
  const int P = g.P, ny = g.ny, N = g.N;
  const int p0 = blockIdx.x * ppc;
  const int b = blockIdx.y;
  if (pb.active && !pb.active[b]) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  pdl_wait_then_release();  // H comes from the nonlinear term
  CN* hb = hn + (size_t)b * 3 * ny * P;
  constexpr int NF = 2 * (MH - 1);
  if constexpr (std::is_same<RN, double>::value && ct_plan_ok(NF)) {
    if (N == NF) {
      // FFT form over the three fields of the tile, coefficients straight to hn
      double2* X = reinterpret_cast<double2*>(smem_raw);  // [3][ny][ppc]
      for (int w = tid; w < 3 * ny * ppc; w += nt) {
        const int pl = w % ppc, fn = w / ppc;
        X[w] = hb[(size_t)fn * P + min(p0 + pl, P - 1)];
      }
      __syncthreads();
      analysis_fft<NF>(X, ppc, ny, P, p0, X + 3 * ny * ppc, t.cheb, t.tw_cheb, hb + p0);
      return;
    }
  }
  // direct sums, one field at a time: thread (mode pl, group gq of 8) forms
  // the coefficients n = gq + 8 k
  constexpr int KN = (2 * MH + 7) / 8;
  CN* col0 = reinterpret_cast<CN*>(smem_raw);  // [ny][ppc]
  const int pl = tid % ppc, gq = tid / ppc;
  const RN* cheb = cheb_table<RN>(t);
  const RN sg = (gq & 1) ? (RN)-1.0 : (RN)1.0;
  for (int f = 0; f < 3; ++f) {
    CN* hf = hb + (size_t)f * ny * P;
    for (int w = tid; w < ny * ppc; w += nt) {
      const int q = w % ppc, n = w / ppc;
      col0[w] = hf[(size_t)n * P + min(p0 + q, P - 1)];
    }
    __syncthreads();
    if (gq < 8) {
      CN acc[KN];
      analysis_sums<RN, KN>(col0 + pl, ppc, N, ny, cheb, gq, 8, sg, acc);
      if (p0 + pl < P) {
#pragma unroll
        for (int k = 0; k < KN; ++k) {
          const int n = gq + 8 * k;
          if (n <= N) hf[(size_t)n * P + p0 + pl] = acc[k];
        }
      }
    }
    __syncthreads();
  }
}

template <typename RN, int MH>
__global__ void __launch_bounds__(64) stage_post_wide_kernel(Grid g, int B, PencilBufs pb, DevTables t,
                                                             const typename cpx<RN>::T* __restrict__ hc,
                                                             StageCoef sc, int ppc) {
  extern __shared__ __align__(16) double sarr[];  // [MH][blockDim.x]
  using CN = typename cpx<RN>::T;
  const int P = g.P, ny = g.ny;
  const int p0 = blockIdx.x * ppc;
  const int b = blockIdx.y;
  if (pb.active && !pb.active[b]) return;
  pdl_wait_then_release();  // the coefficients of H come from the analysis
  const int tid = threadIdx.x;
  const int r = tid & 1, pl = (tid >> 1) % ppc, c = tid / (2 * ppc);
  const int p = p0 + pl;
  if (p >= P) return;  // no barrier in this kernel
  if (p / g.nxh == g.nz / 2) return;  // Nyquist row stays zero
  const CN* Hx = hc + (size_t)b * 3 * ny * P + p;
  const CN* Hy = Hx + (size_t)ny * P;
  const CN* Hz = Hy + (size_t)ny * P;
  const size_t base = 2 * ((size_t)b * ny * P + p) + r;
  const CompT<RN> HGr{reinterpret_cast<RN*>(pb.HGP) + base, 2 * P};
  const CompT<RN> HVr{reinterpret_cast<RN*>(pb.HVP) + base, 2 * P};
  post_solve_noslip<MH, RN, true>(sarr + tid, (int)blockDim.x, c, g, pb, t, sc, b, p, r, Hx, Hy, Hz, P, HGr, HVr);
}

// modes per CTA of the analysis half: 32 with direct sums (256 threads), 8
// with the FP64 FFT form (three fields of the tile in shared memory)
template <typename RN, int MH>
constexpr int post_analysis_ppc() {
  return (std::is_same<RN, double>::value && ct_plan_ok(2 * (MH - 1))) ? 8 : 32;
}

// ---------------------------------------------------------------------------
// per-MH launchers, instantiated in the stage_mh*.cu translation units
// ---------------------------------------------------------------------------
template <typename RN, int MH>
cudaError_t pre_mh(const Grid& g, int B, const PencilBufs& pb, const DevTables& t,
                          typename cpx<RN>::T* q, int ppc, size_t smem, cudaStream_t st) {
  static SmemLimit lim;
  const cudaError_t e = raise_smem_limit(stage_pre_kernel<RN, MH>, &lim, smem);
  if (e != cudaSuccess) return e;
  return launch_pdl_if<sizeof(RN) == 4>(stage_pre_kernel<RN, MH>, dim3((g.P + ppc - 1) / ppc, B), dim3(128), smem,
                                        st, g, B, pb, t, q, ppc);
}

template <typename RN, int MH, int TOP>
cudaError_t post_mh(const Grid& g, int B, const PencilBufs& pb, const DevTables& t,
                           const typename cpx<RN>::T* h, const StageCoef& sc, int ppc, size_t smem,
                           cudaStream_t st) {
  static SmemLimit lim;
  const cudaError_t e = raise_smem_limit(stage_post_kernel<RN, MH, TOP>, &lim, smem);
  if (e != cudaSuccess) return e;
  return launch_pdl_if<sizeof(RN) == 4>(stage_post_kernel<RN, MH, TOP>, dim3((g.P + ppc - 1) / ppc, B),
                                        dim3(8 * post_tile_lanes<TOP>() * ppc), smem, st, g, B, pb, t, h, sc, ppc);
}

template <typename RN, int MH, int TOP>
cudaError_t post_batched_mh(const Grid& g, int B, const PencilBufs& pb, const DevTables& t,
                                   const typename cpx<RN>::T* h, const StageCoef& sc, int ppc, size_t smem,
                                   cudaStream_t st) {
  using CN = typename cpx<RN>::T;
  if constexpr (TOP == 0 && MH > 33) {
    // two launches; the analysis replaces the nodal values of H, which no
    // later kernel of the stage reads, by their coefficients
    constexpr int apc = post_analysis_ppc<RN, MH>();
    const size_t sa = std::is_same<RN, double>::value && apc == 8
                          ? ((size_t)3 * g.ny + 6) * apc * sizeof(double2)
                          : (size_t)g.ny * apc * sizeof(CN);
    const int na = apc == 8 ? 128 : 8 * apc;
    static SmemLimit lim_a, lim_w;
    cudaError_t e = raise_smem_limit(stage_post_analysis_kernel<RN, MH>, &lim_a, sa);
    if (e != cudaSuccess) return e;
    if ((e = raise_smem_limit(stage_post_wide_kernel<RN, MH>, &lim_w, smem)) != cudaSuccess) return e;
    e = launch_pdl_if<sizeof(RN) == 4>(stage_post_analysis_kernel<RN, MH>, dim3((g.P + apc - 1) / apc, B), dim3(na),
                                       sa, st, g, B, pb, t, const_cast<CN*>(h), apc);
    if (e != cudaSuccess) return e;
    return launch_pdl_if<sizeof(RN) == 4>(stage_post_wide_kernel<RN, MH>, dim3((g.P + ppc - 1) / ppc, B),
                                          dim3(4 * ppc), smem, st, g, B, pb, t, h, sc, ppc);
  } else {
    static SmemLimit lim;
    const cudaError_t e = raise_smem_limit(stage_post_batched_kernel<RN, MH, TOP>, &lim, smem);
    if (e != cudaSuccess) return e;
    return launch_pdl_if<sizeof(RN) == 4>(stage_post_batched_kernel<RN, MH, TOP>, dim3((g.P + ppc - 1) / ppc, B),
                                          dim3(4 * ppc), smem, st, g, B, pb, t, h, sc, ppc);
  }
}

}  // namespace chdns

// explicit instantiations of the launchers for one register-array bound MH,
// both node precisions, by kernel form
#define CH_STAGE_PRE(MH)                                                                                       \
  namespace chdns {                                                                                            \
  template cudaError_t pre_mh<double, MH>(const Grid&, int, const PencilBufs&, const DevTables&, double2*, int,  \
                                          size_t, cudaStream_t);                                               \
  template cudaError_t pre_mh<float, MH>(const Grid&, int, const PencilBufs&, const DevTables&, float2*, int,    \
                                         size_t, cudaStream_t);                                                \
  }
#define CH_STAGE_POST_TOP(MH, TOP)                                                                             \
  namespace chdns {                                                                                            \
  template cudaError_t post_mh<double, MH, TOP>(const Grid&, int, const PencilBufs&, const DevTables&,          \
                                                const double2*, const StageCoef&, int, size_t, cudaStream_t);  \
  template cudaError_t post_mh<float, MH, TOP>(const Grid&, int, const PencilBufs&, const DevTables&,           \
                                               const float2*, const StageCoef&, int, size_t, cudaStream_t);    \
  }
#define CH_STAGE_POST_BATCHED_TOP(MH, TOP)                                                                     \
  namespace chdns {                                                                                            \
  template cudaError_t post_batched_mh<double, MH, TOP>(const Grid&, int, const PencilBufs&, const DevTables&,  \
                                                        const double2*, const StageCoef&, int, size_t,         \
                                                        cudaStream_t);                                         \
  template cudaError_t post_batched_mh<float, MH, TOP>(const Grid&, int, const PencilBufs&, const DevTables&,   \
                                                       const float2*, const StageCoef&, int, size_t,           \
                                                       cudaStream_t);                                          \
  }
// no-slip upper wall (TOP = 0) for every bucket; the free-slip top (TOP = 1)
// is instantiated for MH <= 33 (ny <= 65) in translation units of its own
#define CH_STAGE_POST(MH) CH_STAGE_POST_TOP(MH, 0)
#define CH_STAGE_POST_BATCHED(MH) CH_STAGE_POST_BATCHED_TOP(MH, 0)
#define CH_STAGE_INSTANTIATE(MH) CH_STAGE_PRE(MH) CH_STAGE_POST(MH) CH_STAGE_POST_BATCHED(MH)
#define CH_STAGE_INSTANTIATE_OPEN(MH) CH_STAGE_POST_TOP(MH, 1) CH_STAGE_POST_BATCHED_TOP(MH, 1)
