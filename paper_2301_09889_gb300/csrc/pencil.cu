// Wall-normal (Chebyshev) work of one Runge-Kutta stage, one thread per
// (environment, Fourier mode, symmetry class), plus the small kernels of the
// environment step (action, observation, wall shear, reward).
//
// Symmetry classes.  Every wall-normal operator of the velocity-vorticity
// system (D, D^2, the tau rows, the wall conditions split into sums and
// differences) maps even Chebyshev coefficients to even ones or to odd ones
// in a fixed pattern, so a mode splits into two independent halves:
//   class 0: even v, odd  omega_y  (u, w odd;  omega_x, omega_z even)
//   class 1: odd  v, even omega_y  (u, w even; omega_x, omega_z odd)
// One thread owns one half and never exchanges data with the other.
//
// Chebyshev conventions: f(y) = sum_n a_n T_n(y), nodes y_j = cos(pi j / N).
// Derivative recurrence (coefficient space): c_m b_m = b_{m+2} + 2 (m+1) a_{m+1}
// with c_0 = 2, c_m = 1 otherwise, walked from m = N down to 0.
#include <mutex>

#include "../../include/channel_dns.h"
#include "common.cuh"
#include "internal.h"

namespace chdns {

// ---------------------------------------------------------------------------
// Chebyshev-tau Dirichlet problem (D^2 - lam) f = r, split by parity.
//
// For n >= 2 the tau rows are equivalent to the quasi-tridiagonal rows
//   -lam c_{n-2}/(4n(n-1)) f_{n-2} + (1 + lam b_n/(2(n^2-1))) f_n
//   - lam b_{n+2}/(4n(n+1)) f_{n+2}
//     = c_{n-2}/(4n(n-1)) r_{n-2} - b_n/(2(n^2-1)) r_n + b_{n+2}/(4n(n+1)) r_{n+2}
// (b_m = 1 for m <= N-2, else 0: the two highest rows of r are dropped), obtained
// by integrating D^2 f = r + lam f twice.  With parity index i (n = 2i + sig) the
// rows i >= 1 are tridiagonal; the wall row sum_i f_i = s closes the system.
// Elimination from the bottom gives f_i = a_i + b_i f_{i-1}; all f_i are then
// affine in f_0, which the wall row fixes.  The lam-dependent factors
// e_i = 1/den_i, h_i = U_i/den_i, b_i = -L_i/den_i, Q_i = prod b and 1/sum Q
// are precomputed per mode and stage.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double tau_cA(int n) { return (n == 2 ? 2.0 : 1.0) / (4.0 * n * (n - 1)); }
__device__ __forceinline__ double tau_cB(int n, int N) { return n <= N - 2 ? 1.0 / (2.0 * ((double)n * n - 1.0)) : 0.0; }
__device__ __forceinline__ double tau_cC(int n, int N) { return n + 2 <= N - 2 ? 1.0 / (4.0 * n * (n + 1)) : 0.0; }

struct TabGlobal {
  const double* base;  // element (field f, index i) at base[(f * Mh + i) * P]
  int Mh, P;
  __device__ double e(int i) const { return base[(size_t)(0 * Mh + i) * P]; }
  __device__ double h(int i) const { return base[(size_t)(1 * Mh + i) * P]; }
  __device__ double b(int i) const { return base[(size_t)(2 * Mh + i) * P]; }
  __device__ double Q(int i) const { return base[(size_t)(3 * Mh + i) * P]; }
};

struct TabLocal {
  const double *pe, *ph, *pb, *pQ;
  __device__ double e(int i) const { return pe[i]; }
  __device__ double h(int i) const { return ph[i]; }
  __device__ double b(int i) const { return pb[i]; }
  __device__ double Q(int i) const { return pQ[i]; }
};

// r[i] = r_{2i+sig}; f[i] receives f_{2i+sig}.  r and f must not alias.
template <class Tab>
__device__ void tau_solve(int N, int sig, const double2* r, double2* f, const Tab& T, double isq, double2 s) {
  const int M = (N - sig) / 2 + 1;
  double2 anext = mk(0.0, 0.0);
  for (int i = M - 1; i >= 1; --i) {
    const int n = 2 * i + sig;
    double2 R = tau_cA(n) * r[i - 1] - tau_cB(n, N) * r[i];
    if (i + 1 < M) R = R + tau_cC(n, N) * r[i + 1];
    const double2 a = T.e(i) * R - T.h(i) * anext;
    f[i] = a;
    anext = a;
  }
  double2 Pp = mk(0.0, 0.0), sum = mk(0.0, 0.0);
  for (int i = 1; i < M; ++i) {
    Pp = f[i] + T.b(i) * Pp;
    f[i] = Pp;
    sum = sum + Pp;
  }
  const double2 f0 = isq * (s - sum);
  f[0] = f0;
  for (int i = 1; i < M; ++i) f[i] = f[i] + T.Q(i) * f0;
}

// on-the-fly factorisation of one parity (for the stateless entry point)
__device__ void tau_factor(int N, int sig, double lam, double* e, double* h, double* b, double* Q, double* isq) {
  const int M = (N - sig) / 2 + 1;
  double bnext = 0.0;
  e[0] = h[0] = b[0] = 0.0;
  for (int i = M - 1; i >= 1; --i) {
    const int n = 2 * i + sig;
    const double L = -lam * tau_cA(n);
    const double Dg = 1.0 + lam * tau_cB(n, N);
    const double U = (i + 1 < M) ? -lam * tau_cC(n, N) : 0.0;
    const double den = Dg + U * bnext;
    e[i] = 1.0 / den;
    h[i] = U / den;
    b[i] = -L / den;
    bnext = b[i];
  }
  Q[0] = 1.0;
  double sq = 1.0;
  for (int i = 1; i < M; ++i) {
    Q[i] = b[i] * Q[i - 1];
    sq += Q[i];
  }
  *isq = 1.0 / sq;
}

// ---------------------------------------------------------------------------
// recover: (v, omega_y, U, W) coefficients -> coefficients of
// u, v, w, omega_x, omega_y, omega_z.
//   u = (i kx Dv - i kz g)/k^2, w = (i kz Dv + i kx g)/k^2,
//   omega_x = Dw - i kz v, omega_z = i kx v - Du;  mean mode: u = U, w = W,
//   omega_x = DW, omega_z = -DU.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) recover_kernel(Grid g, int B, PencilBufs pb, DevTables t) {
  const int P = g.P, ny = g.ny, N = g.N;
  const long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (tid >= 2L * P * B) return;
  const int p = (int)(tid % P);
  const int c = (int)((tid / P) % 2);
  const int b = (int)(tid / (2L * P));
  const int row = p / g.nxh, ix = p % g.nxh;
  const size_t fo = (size_t)b * ny * P + p;
  double2* out = pb.C6 + (size_t)b * 6 * ny * P + p;  // field f, coefficient n: out[(f*ny + n)*P]
  auto W6 = [&](int f, int n, double2 v) { out[((size_t)f * ny + n) * P] = v; };
  const double2 zero = mk(0.0, 0.0);

  if (row == g.nz / 2) {  // Nyquist row: all zero
    for (int n = N; n >= 0; --n)
      if ((n & 1) == c)
        for (int f = 0; f < 6; ++f) W6(f, n, zero);
    return;
  }
  if (p == 0) {
    // class c: u = U and w = W on parity 1-c, omega_x = DW, omega_z = -DU on parity c
    const double* U = pb.UM + (size_t)b * ny;
    const double* Wm = pb.WM + (size_t)b * ny;
    double du = 0.0, dw = 0.0, unext = 0.0, wnext = 0.0;
    for (int n = N; n >= 0; --n) {
      if ((n & 1) == 1 - c) {
        const double un = U[n], wn = Wm[n];
        W6(0, n, mk(un, 0.0));
        W6(1, n, zero);
        W6(2, n, mk(wn, 0.0));
        W6(4, n, zero);
        unext = un;
        wnext = wn;
      } else {
        double t1 = du + 2.0 * (n + 1) * unext;
        double t2 = dw + 2.0 * (n + 1) * wnext;
        du = (n == 0) ? 0.5 * t1 : t1;
        dw = (n == 0) ? 0.5 * t2 : t2;
        W6(1, n, zero);
        W6(3, n, mk(dw, 0.0));
        W6(5, n, mk(-du, 0.0));
        // u, w, omega_y on this parity belong to the other class
      }
    }
    return;
  }
  const double kx = t.kx[ix], kz = t.kz[row];
  const double ik2 = 1.0 / (kx * kx + kz * kz);
  double2 dv = zero, d2v = zero, dg = zero, vnext = zero, gnext = zero;
  for (int n = N; n >= 0; --n) {
    if ((n & 1) == 1 - c) {
      // Dv_n from v_{n+1}; g_n lives on this parity
      const double2 t1 = dv + (2.0 * (n + 1)) * vnext;
      dv = (n == 0) ? 0.5 * t1 : t1;
      const double2 gn = pb.G[fo + (size_t)n * P];
      const double2 u = ik2 * (imul(kx, dv) - imul(kz, gn));
      const double2 w = ik2 * (imul(kz, dv) + imul(kx, gn));
      W6(0, n, u);
      W6(2, n, w);
      W6(4, n, gn);
      gnext = gn;
    } else {
      // D^2 v_n from Dv_{n+1}; Dg_n from g_{n+1}; v_n lives on this parity
      const double2 t1 = d2v + (2.0 * (n + 1)) * dv;
      const double2 t2 = dg + (2.0 * (n + 1)) * gnext;
      d2v = (n == 0) ? 0.5 * t1 : t1;
      dg = (n == 0) ? 0.5 * t2 : t2;
      const double2 vn = pb.V[fo + (size_t)n * P];
      const double2 du = ik2 * (imul(kx, d2v) - imul(kz, dg));
      const double2 dw = ik2 * (imul(kz, d2v) + imul(kx, dg));
      W6(1, n, vn);
      W6(3, n, dw - imul(kz, vn));
      W6(5, n, imul(kx, vn) - du);
      vnext = vn;
    }
  }
}

// ---------------------------------------------------------------------------
// Chebyshev synthesis: node values f_j = sum_n a_n cos(pi n j / N) of
// `nfields` fields.  cos(pi n (N-j)/N) = (-1)^n cos(pi n j / N), so the even
// and odd partial sums E_j, O_j give f_j = E + O and f_{N-j} = E - O.
// CTA: 32 modes x 8 node groups; grid (ceil(P/32), nfields, B).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) synth_kernel(int ny, int P, int nfields, const double2* coef,
                                                    double2* out, const double* cheb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* sc = reinterpret_cast<double2*>(smem_raw);  // [ny][32]
  const int pl = threadIdx.x % 32, jg = threadIdx.x / 32;
  const int p0 = blockIdx.x * 32;
  const size_t fo = ((size_t)blockIdx.z * nfields + blockIdx.y) * ny * P;
  const double2* src = coef + fo;
  for (int idx = threadIdx.x; idx < ny * 32; idx += blockDim.x) {
    const int n = idx / 32, pp = idx % 32;
    sc[idx] = (p0 + pp < P) ? src[(size_t)n * P + p0 + pp] : mk(0.0, 0.0);
  }
  __syncthreads();
  const int N = ny - 1;
  const int p = p0 + pl;
  if (p >= P) return;
  double2* dst = out + fo + p;
  for (int j = jg; 2 * j <= N; j += 8) {
    const double* crow = cheb + (size_t)j * ny;
    double2 E = mk(0.0, 0.0), O = mk(0.0, 0.0);
    for (int n = 0; n <= N; n += 2) E = E + crow[n] * sc[n * 32 + pl];
    for (int n = 1; n <= N; n += 2) O = O + crow[n] * sc[n * 32 + pl];
    dst[(size_t)j * P] = E + O;
    if (N - j != j) dst[(size_t)(N - j) * P] = E - O;
  }
}

// ---------------------------------------------------------------------------
// Chebyshev analysis: a_n = 2/(N cb_n) sum_j f_j cos(pi n j / N) / cb_j with
// cb_0 = cb_N = 2, else 1.  Node pairs (j, N-j) are folded into
// e_j = (f_j + f_{N-j})/cb_j for even n and o_j = (f_j - f_{N-j})/cb_j for odd n.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) analysis_kernel(int ny, int P, int nfields, const double2* nodes,
                                                       double2* coef, const double* cheb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = ny - 1;
  const int H = N / 2 + 1;
  double2* se = reinterpret_cast<double2*>(smem_raw);  // [H][32]
  double2* so = se + H * 32;                            // [H][32]
  const int pl = threadIdx.x % 32, ng = threadIdx.x / 32;
  const int p0 = blockIdx.x * 32;
  const size_t fo = ((size_t)blockIdx.z * nfields + blockIdx.y) * ny * P;
  const double2* src = nodes + fo;
  for (int idx = threadIdx.x; idx < H * 32; idx += blockDim.x) {
    const int j = idx / 32, pp = idx % 32;
    double2 ev = mk(0.0, 0.0), od = mk(0.0, 0.0);
    if (p0 + pp < P) {
      const double2 fj = src[(size_t)j * P + p0 + pp];
      if (N - j != j) {
        const double2 fm = src[(size_t)(N - j) * P + p0 + pp];
        const double w = (j == 0) ? 0.5 : 1.0;
        ev = w * (fj + fm);
        od = w * (fj - fm);
      } else {
        ev = fj;
      }
    }
    se[idx] = ev;
    so[idx] = od;
  }
  __syncthreads();
  const int p = p0 + pl;
  if (p >= P) return;
  double2* dst = coef + fo + p;
  const double s0 = 2.0 / N;
  for (int n = ng; n <= N; n += 8) {
    const double* crow = cheb + (size_t)n * ny;
    const double2* sv = (n & 1) ? so : se;
    double2 acc = mk(0.0, 0.0);
    for (int j = 0; j < H; ++j) acc = acc + crow[j] * sv[j * 32 + pl];
    const double cbn = (n == 0 || n == N) ? 2.0 : 1.0;
    dst[(size_t)n * P] = (s0 / cbn) * acc;
  }
}

// ---------------------------------------------------------------------------
// implicit part of one stage: RHS assembly and the tau solves.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(64) solve_kernel(Grid g, int B, PencilBufs pb, DevTables t, StageCoef sc) {
  const int P = g.P, ny = g.ny, N = g.N;
  const long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (tid >= 2L * P * B) return;
  const int p = (int)(tid % P);
  const int c = (int)((tid / P) % 2);
  const int b = (int)(tid / (2L * P));
  const int row = p / g.nxh, ix = p % g.nxh;
  if (row == g.nz / 2) return;  // Nyquist row stays zero
  const size_t fo = (size_t)b * ny * P + p;
  const double2* Hx = pb.HC + (size_t)b * 3 * ny * P + p;
  const double2* Hy = Hx + (size_t)ny * P;
  const double2* Hz = Hy + (size_t)ny * P;
  const double ibdn = 1.0 / (sc.beta * sc.dt * sc.nu);
  const double adn = sc.alpha * sc.dt * sc.nu;
  const int Mh = t.tau.Mh;
  double2 rr[kMaxHalf], ff[kMaxHalf];
  const double2 zero = mk(0.0, 0.0);

  if (p == 0) {
    // mean flow: class c owns parity c of U and W
    const int s = c;
    double* U = pb.UM + (size_t)b * ny;
    double* Wm = pb.WM + (size_t)b * ny;
    double* HXP = pb.HXP + (size_t)b * ny;
    double* HZP = pb.HZP + (size_t)b * ny;
    double du = 0.0, d2u = 0.0, unext = 0.0, dw = 0.0, d2w = 0.0, wnext = 0.0;
    double2 rw[kMaxHalf];
    for (int n = N; n >= 0; --n) {
      if ((n & 1) != s) {
        const double t1 = du + 2.0 * (n + 1) * unext;
        const double t2 = dw + 2.0 * (n + 1) * wnext;
        du = (n == 0) ? 0.5 * t1 : t1;
        dw = (n == 0) ? 0.5 * t2 : t2;
      } else {
        const double t1 = d2u + 2.0 * (n + 1) * du;
        const double t2 = d2w + 2.0 * (n + 1) * dw;
        d2u = (n == 0) ? 0.5 * t1 : t1;
        d2w = (n == 0) ? 0.5 * t2 : t2;
        const double un = U[n], wn = Wm[n];
        const double hx = Hx[(size_t)n * P].x, hz = Hz[(size_t)n * P].x;
        const double hxp = HXP[n], hzp = HZP[n];
        HXP[n] = hx;
        HZP[n] = hz;
        const double ru = -ibdn * (un + adn * d2u + sc.dt * (sc.gamma * hx + sc.zeta * hxp));
        const double rwv = -ibdn * (wn + adn * d2w + sc.dt * (sc.gamma * hz + sc.zeta * hzp));
        rr[(n - s) / 2] = mk(ru, 0.0);
        rw[(n - s) / 2] = mk(rwv, 0.0);
        unext = un;
        wnext = wn;
      }
    }
    const size_t hb = (size_t)((sc.k * 2 + s) * 4) * Mh * P;
    const TabGlobal T{t.tau.helm + hb, Mh, P};
    const double isq = t.tau.helm_isq[(size_t)(sc.k * 2 + s) * P];
    const int M = (N - s) / 2 + 1;
    tau_solve(N, s, rr, ff, T, isq, zero);
    if (s == 0) {
      double flux = 0.0;
      for (int i = 0; i < M; ++i) {
        const int n = 2 * i;
        flux += 2.0 / (1.0 - (double)n * n) * ff[i].x;
      }
      const double fc = (sc.flux - flux) * t.tau.u1_iflux[sc.k];
      for (int i = 0; i < M; ++i) U[2 * i] = ff[i].x + fc * t.tau.u1[(size_t)sc.k * ny + 2 * i];
    } else {
      for (int i = 0; i < M; ++i) U[2 * i + 1] = ff[i].x;
    }
    tau_solve(N, s, rw, ff, T, isq, zero);
    for (int i = 0; i < M; ++i) Wm[2 * i + s] = ff[i].x;
    return;
  }

  const double kx = t.kx[ix], kz = t.kz[row], k2 = kx * kx + kz * kz;
  const int sv = c, sg = 1 - c;

  // ---- wall-normal vorticity (parity sg): (D^2 - lam) g^k = r_g, g = 0 at both walls
  {
    double2 dg = zero, d2g = zero, gnext = zero;
    for (int n = N; n >= 0; --n) {
      if ((n & 1) == sv) {
        const double2 t1 = dg + (2.0 * (n + 1)) * gnext;
        dg = (n == 0) ? 0.5 * t1 : t1;
      } else {
        const double2 t1 = d2g + (2.0 * (n + 1)) * dg;
        d2g = (n == 0) ? 0.5 * t1 : t1;
        const size_t o = fo + (size_t)n * P;
        const double2 gn = pb.G[o];
        const double2 hx = Hx[(size_t)n * P], hz = Hz[(size_t)n * P];
        const double2 hg = imul(kz, hx) - imul(kx, hz);
        const double2 hgp = pb.HGP[o];
        pb.HGP[o] = hg;
        const double2 lap = d2g - k2 * gn;
        rr[(n - sg) / 2] = (-ibdn) * (gn + adn * lap + sc.dt * (sc.gamma * hg + sc.zeta * hgp));
        gnext = gn;
      }
    }
    const size_t hb = (size_t)((sc.k * 2 + sg) * 4) * Mh * P + p;
    const TabGlobal T{t.tau.helm + hb, Mh, P};
    const double isq = t.tau.helm_isq[(size_t)(sc.k * 2 + sg) * P + p];
    tau_solve(N, sg, rr, ff, T, isq, zero);
    const int M = (N - sg) / 2 + 1;
    for (int i = 0; i < M; ++i) pb.G[fo + (size_t)(2 * i + sg) * P] = ff[i];
  }

  // ---- wall-normal velocity (parity sv): phi = lap v
  {
    double2 dv = zero, d2v = zero, dphi = zero, d2phi = zero, dtt = zero;
    double2 vnext = zero, phinext = zero, tnext = zero;
    for (int n = N; n >= 0; --n) {
      if ((n & 1) == sg) {
        const double2 t1 = dv + (2.0 * (n + 1)) * vnext;
        const double2 t2 = dphi + (2.0 * (n + 1)) * phinext;
        dv = (n == 0) ? 0.5 * t1 : t1;
        dphi = (n == 0) ? 0.5 * t2 : t2;
        const double2 hx = Hx[(size_t)n * P], hz = Hz[(size_t)n * P];
        tnext = imul(kx, hx) + imul(kz, hz);
      } else {
        const double2 t0 = dtt + (2.0 * (n + 1)) * tnext;
        const double2 t1 = d2v + (2.0 * (n + 1)) * dv;
        const double2 t2 = d2phi + (2.0 * (n + 1)) * dphi;
        dtt = (n == 0) ? 0.5 * t0 : t0;
        d2v = (n == 0) ? 0.5 * t1 : t1;
        d2phi = (n == 0) ? 0.5 * t2 : t2;
        const size_t o = fo + (size_t)n * P;
        const double2 vn = pb.V[o];
        const double2 phin = d2v - k2 * vn;
        const double2 hv = (-k2) * Hy[(size_t)n * P] - dtt;
        const double2 hvp = pb.HVP[o];
        pb.HVP[o] = hv;
        rr[(n - sv) / 2] =
            (-ibdn) * (phin + adn * (d2phi - k2 * phin) + sc.dt * (sc.gamma * hv + sc.zeta * hvp));
        vnext = vn;
        phinext = phin;
      }
    }
    // phi_p: (D^2 - lam) phi_p = r_phi, phi_p = 0 at both walls
    const size_t hb = (size_t)((sc.k * 2 + sv) * 4) * Mh * P + p;
    const TabGlobal TH{t.tau.helm + hb, Mh, P};
    tau_solve(N, sv, rr, ff, TH, t.tau.helm_isq[(size_t)(sc.k * 2 + sv) * P + p], zero);
    // v_p: (D^2 - k^2) v_p = phi_p, v_p(+1) = 0, v_p(-1) = v_w
    const size_t vo = (size_t)b * P + p;
    const double2 vw = pb.vw_old[vo] + sc.theta * (pb.vw_new[vo] - pb.vw_old[vo]);
    const double2 s = (sv == 0) ? 0.5 * vw : (-0.5) * vw;
    const TabGlobal TP{t.tau.pois + (size_t)(sv * 4) * Mh * P + p, Mh, P};
    tau_solve(N, sv, ff, rr, TP, t.tau.pois_isq[(size_t)sv * P + p], s);
    // influence-matrix correction: Dv(+-1) = 0
    const int M = (N - sv) / 2 + 1;
    double2 dp = zero;
    for (int i = 0; i < M; ++i) {
      const int n = 2 * i + sv;
      dp = dp + (double)(n * n) * rr[i];
    }
    const double2 cI = (-t.tau.vh_idv[(size_t)(sc.k * 2 + sv) * P + p]) * dp;
    const double* vh = t.tau.vh + (size_t)sc.k * ny * P + p;
    for (int i = 0; i < M; ++i) {
      const int n = 2 * i + sv;
      pb.V[fo + (size_t)n * P] = rr[i] + vh[(size_t)n * P] * cI;
    }
  }
}

// ---------------------------------------------------------------------------
// wall shear of the lower wall: tau_w = nu sum_n U_n T_n'(-1), T_n'(-1) = (-1)^(n+1) n^2
// one warp per environment, fixed summation order
// ---------------------------------------------------------------------------
__global__ void wall_shear_kernel(int ny, int B, const double* UM, double nu, double* acc) {
  const int b = blockIdx.x;
  if (b >= B) return;
  const int lane = threadIdx.x;
  double s = 0.0;
  for (int n = lane; n < ny; n += 32) {
    const double d = (double)n * n * ((n & 1) ? 1.0 : -1.0);
    s += d * UM[(size_t)b * ny + n];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) acc[b] += nu * s;
}

// ---------------------------------------------------------------------------
// sensing plane: Fourier coefficients of u and v at node js (and, for
// opposition control, the wall spectrum -alpha v(y_s) with the mean removed,
// paper Sec. 4.1)
// ---------------------------------------------------------------------------
__global__ void sense_kernel(Grid g, int B, PencilBufs pb, DevTables t, int js, double alpha, int opposition) {
  const int P = g.P, ny = g.ny, N = g.N;
  const long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (tid >= (long)P * B) return;
  const int p = (int)(tid % P);
  const int b = (int)(tid / P);
  const int row = p / g.nxh, ix = p % g.nxh;
  const double* cj = t.cheb + (size_t)js * ny;
  double2 us = mk(0.0, 0.0), vs = mk(0.0, 0.0);
  if (row != g.nz / 2) {
    if (p == 0) {
      double s = 0.0;
      for (int n = 0; n <= N; ++n) s += cj[n] * pb.UM[(size_t)b * ny + n];
      us = mk(s, 0.0);
    } else {
      const size_t fo = (size_t)b * ny * P + p;
      double2 d1 = mk(0.0, 0.0), d2 = mk(0.0, 0.0);  // Dv_{n+1}, Dv_{n+2}
      double2 vnext = mk(0.0, 0.0);
      double2 dvs = mk(0.0, 0.0), gs = mk(0.0, 0.0);
      for (int n = N; n >= 0; --n) {
        const double2 tt = d2 + (2.0 * (n + 1)) * vnext;
        const double2 dn = (n == 0) ? 0.5 * tt : tt;
        const double2 vn = pb.V[fo + (size_t)n * P];
        const double2 gn = pb.G[fo + (size_t)n * P];
        vs = vs + cj[n] * vn;
        gs = gs + cj[n] * gn;
        dvs = dvs + cj[n] * dn;
        d2 = d1;
        d1 = dn;
        vnext = vn;
      }
      const double kx = t.kx[ix], kz = t.kz[row];
      const double ik2 = 1.0 / (kx * kx + kz * kz);
      us = ik2 * (imul(kx, dvs) - imul(kz, gs));
    }
  }
  if (opposition) {
    pb.vw_new[(size_t)b * P + p] = (p == 0) ? mk(0.0, 0.0) : (-alpha) * vs;
  } else {
    pb.planes[((size_t)b * 2 + 0) * P + p] = us;
    pb.planes[((size_t)b * 2 + 1) * P + p] = vs;
  }
}

// ---------------------------------------------------------------------------
// observation planes: unpadded inverse transform of the two sensing-plane
// spectra, f(x_a, z_b) = Re sum_kz F[kz,0] e^{i kz z} + 2 Re sum_{kx>0} F e^{i(kx x + kz z)}
// one CTA per (environment, field)
// ---------------------------------------------------------------------------
__global__ void obs_kernel(int nx, int nz, int nxh, const double2* planes, const double2* tw_nx,
                           const double2* tw_nz, double* out, size_t out_stride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* tmp = reinterpret_cast<double2*>(smem_raw);  // [nz][nxh]
  const int b = blockIdx.y, f = blockIdx.x;
  const int P = nz * nxh;
  const double2* F = planes + ((size_t)b * 2 + f) * P;
  for (int w = threadIdx.x; w < nz * nxh; w += blockDim.x) {
    const int i = w % nxh, zb = w / nxh;
    double2 acc = mk(0.0, 0.0);
    for (int row = 0; row < nz; ++row) {
      if (row == nz / 2) continue;
      const int m = row < nz / 2 ? row : row - nz;
      int e = (m * zb) % nz;
      if (e < 0) e += nz;
      acc = acc + cmul(F[row * nxh + i], tw_nz[e]);
    }
    tmp[zb * nxh + i] = acc;
  }
  __syncthreads();
  double* o = out + (size_t)b * out_stride + (size_t)f * nz * nx;
  for (int w = threadIdx.x; w < nz * nx; w += blockDim.x) {
    const int xa = w % nx, zb = w / nx;
    double s = 0.0;
    for (int i = 1; i < nxh; ++i) {
      const double2 tw = tw_nx[(i * xa) % nx];
      const double2 v = tmp[zb * nxh + i];
      s += v.x * tw.x - v.y * tw.y;
    }
    o[(size_t)zb * nx + xa] = tmp[zb * nxh].x + 2.0 * s;
  }
}

// ---------------------------------------------------------------------------
// wall action -> wall spectrum: clip to [-u_tau, u_tau], remove the plane
// mean (zero net mass flux), forward transform of the kept modes; the mean
// mode and the Nyquist row are zero.  One CTA per environment.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) action_kernel(int nx, int nz, int nxh, const double* act, double u_tau,
                                                     const double2* tw_nx, const double2* tw_nz, double2* vw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* a = reinterpret_cast<double*>(smem_raw);          // [nz][nx]
  double2* tx = reinterpret_cast<double2*>(a + nz * nx);    // [nz][nxh]
  __shared__ double red[256];
  const int b = blockIdx.x;
  const double* src = act + (size_t)b * nz * nx;
  double s = 0.0;
  for (int w = threadIdx.x; w < nz * nx; w += blockDim.x) {
    const double v = fmin(fmax(src[w], -u_tau), u_tau);
    a[w] = v;
    s += v;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double mean = red[0] / (double)(nz * nx);
  for (int w = threadIdx.x; w < nz * nx; w += blockDim.x) a[w] -= mean;
  __syncthreads();
  for (int w = threadIdx.x; w < nz * nxh; w += blockDim.x) {
    const int i = w % nxh, zb = w / nxh;
    double2 acc = mk(0.0, 0.0);
    for (int xa = 0; xa < nx; ++xa) acc = acc + a[zb * nx + xa] * cconj(tw_nx[(i * xa) % nx]);
    tx[zb * nxh + i] = acc;
  }
  __syncthreads();
  const double sc = 1.0 / (double)(nx * nz);
  for (int w = threadIdx.x; w < nz * nxh; w += blockDim.x) {
    const int i = w % nxh, row = w / nxh;
    double2 acc = mk(0.0, 0.0);
    if (row != nz / 2 && w != 0) {
      const int m = row < nz / 2 ? row : row - nz;
      for (int zb = 0; zb < nz; ++zb) {
        int e = (m * zb) % nz;
        if (e < 0) e += nz;
        acc = acc + cmul(tx[zb * nxh + i], cconj(tw_nz[e]));
      }
      acc = sc * acc;
    }
    vw[(size_t)b * nz * nxh + w] = acc;
  }
}

__global__ void finalize_kernel(int B, const double* acc, double inv_steps, double tau_ref, double* out,
                                size_t out_stride, size_t out_offset) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const double tau = acc[b] * inv_steps;
  out[(size_t)b * out_stride + out_offset] = tau;
  out[(size_t)b * out_stride + out_offset + 1] = 1.0 - tau / tau_ref;
}

// stateless tau problems: one thread per (problem, parity)
__global__ void tau_helmholtz_kernel(int ny, int M, const double* lam, const double2* r, const double2* top,
                                     const double2* bot, double2* f) {
  const long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (tid >= 2L * M) return;
  const int m = (int)(tid / 2), sig = (int)(tid % 2);
  const int N = ny - 1;
  double e[kMaxHalf], h[kMaxHalf], bb[kMaxHalf], Q[kMaxHalf], isq;
  tau_factor(N, sig, lam[m], e, h, bb, Q, &isq);
  const int Mp = (N - sig) / 2 + 1;
  double2 rr[kMaxHalf], ff[kMaxHalf];
  for (int i = 0; i < Mp; ++i) rr[i] = r[(size_t)m * ny + 2 * i + sig];
  const double2 s = sig == 0 ? 0.5 * (top[m] + bot[m]) : 0.5 * (top[m] - bot[m]);
  tau_solve(N, sig, rr, ff, TabLocal{e, h, bb, Q}, isq, s);
  for (int i = 0; i < Mp; ++i) f[(size_t)m * ny + 2 * i + sig] = ff[i];
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_recover(const Grid& g, int B, const PencilBufs& pb, const DevTables& t, cudaStream_t st) {
  const long n = 2L * g.P * B;
  recover_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(g, B, pb, t);
  return cudaGetLastError();
}

cudaError_t launch_synth(const Grid& g, int B, const double2* coef, double2* out, const double* cheb,
                         int nfields, cudaStream_t st) {
  const size_t smem = (size_t)g.ny * 32 * sizeof(double2);
  static bool cfg = false;
  if (!cfg) {
    cudaError_t e = cudaFuncSetAttribute(synth_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    cfg = true;
  }
  dim3 grid((g.P + 31) / 32, nfields, B);
  synth_kernel<<<grid, 256, smem, st>>>(g.ny, g.P, nfields, coef, out, cheb);
  return cudaGetLastError();
}

cudaError_t launch_analysis(const Grid& g, int B, const double2* nodes, double2* coef, const double* cheb,
                            int nfields, cudaStream_t st) {
  const int H = g.N / 2 + 1;
  const size_t smem = (size_t)2 * H * 32 * sizeof(double2);
  static bool cfg = false;
  if (!cfg) {
    cudaError_t e = cudaFuncSetAttribute(analysis_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    cfg = true;
  }
  dim3 grid((g.P + 31) / 32, nfields, B);
  analysis_kernel<<<grid, 256, smem, st>>>(g.ny, g.P, nfields, nodes, coef, cheb);
  return cudaGetLastError();
}

cudaError_t launch_solve(const Grid& g, int B, const PencilBufs& pb, const DevTables& t, const StageCoef& sc,
                         cudaStream_t st) {
  const long n = 2L * g.P * B;
  solve_kernel<<<(unsigned)((n + 63) / 64), 64, 0, st>>>(g, B, pb, t, sc);
  return cudaGetLastError();
}

cudaError_t launch_wall_shear(const Grid& g, int B, const double* UM, double nu, double* acc, cudaStream_t st) {
  wall_shear_kernel<<<B, 32, 0, st>>>(g.ny, B, UM, nu, acc);
  return cudaGetLastError();
}

cudaError_t launch_sense(const Grid& g, int B, const PencilBufs& pb, const DevTables& t, int js, double alpha,
                         int opposition, cudaStream_t st) {
  const long n = (long)g.P * B;
  sense_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(g, B, pb, t, js, alpha, opposition);
  return cudaGetLastError();
}

cudaError_t launch_obs(const Grid& g, int B, const double2* planes, const DevTables& t, double* out,
                       size_t out_stride, cudaStream_t st) {
  const size_t smem = (size_t)g.nz * g.nxh * sizeof(double2);
  static bool cfg = false;
  if (!cfg) {
    cudaError_t e = cudaFuncSetAttribute(obs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    cfg = true;
  }
  obs_kernel<<<dim3(2, B), 256, smem, st>>>(g.nx, g.nz, g.nxh, planes, t.tw_nx, t.tw_nz, out, out_stride);
  return cudaGetLastError();
}

cudaError_t launch_action(const Grid& g, int B, const double* act, double u_tau, const DevTables& t, double2* vw,
                          cudaStream_t st) {
  const size_t smem = (size_t)g.nz * g.nx * sizeof(double) + (size_t)g.nz * g.nxh * sizeof(double2);
  static bool cfg = false;
  if (!cfg) {
    cudaError_t e = cudaFuncSetAttribute(action_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    cfg = true;
  }
  action_kernel<<<B, 256, smem, st>>>(g.nx, g.nz, g.nxh, act, u_tau, t.tw_nx, t.tw_nz, vw);
  return cudaGetLastError();
}

cudaError_t launch_finalize(int B, const double* acc, double inv_steps, double tau_ref, double* out,
                            size_t out_stride, size_t out_offset, cudaStream_t st) {
  finalize_kernel<<<(B + 127) / 128, 128, 0, st>>>(B, acc, inv_steps, tau_ref, out, out_stride, out_offset);
  return cudaGetLastError();
}

cudaError_t launch_tau_helmholtz(int ny, int M, const double* lam, const double2* r, const double2* top,
                                 const double2* bot, double2* f, cudaStream_t st) {
  const long n = 2L * M;
  tau_helmholtz_kernel<<<(unsigned)((n + 63) / 64), 64, 0, st>>>(ny, M, lam, r, top, bot, f);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the stateless tau entry point.
//
// tau_helmholtz_kernel above keeps each problem's factorisation and work
// vectors (about 6.5 KB per thread) in local memory, which the CUDA driver
// allocates and may have to grow at launch time.  Some callers cannot let
// anything allocate device memory: a control loop with a fixed real-time
// budget (cudaMalloc and a driver-side resize can block for milliseconds and
// synchronise the device), a process whose device memory is already fully
// handed to another allocator's pool, or a host framework that only lends out
// buffers it owns.  For them the work vectors live in one file-scope array
// below, sized once when the library is loaded.
// ---------------------------------------------------------------------------
}  // namespace chdns

// 16 MiB of doubles, held by every GPU that loads the library until the
// process exits.  Shared by all calls; a call writes every slot it reads, so
// nothing has to start at zero.
constexpr size_t kNoAllocScratchDoubles = (size_t)2 << 20;
static __device__ __align__(256) double g_tau_noalloc_scratch[kNoAllocScratchDoubles];

namespace chdns {

__global__ void tau_helmholtz_noalloc_kernel(int ny, int M, int mpad, const double* lam, const double2* r,
                                             const double2* top, const double2* bot, double2* f,
                                             double* scratch) {
  const long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (tid >= 2L * M) return;
  const int m = (int)(tid / 2), sig = (int)(tid % 2);
  const int N = ny - 1;
  // slot layout: e, h, b, Q (mpad doubles each), then r and f (mpad complex each)
  double* base = scratch + (size_t)tid * 8 * mpad;
  double* e = base;
  double* h = base + mpad;
  double* bb = base + 2 * mpad;
  double* Q = base + 3 * mpad;
  double2* rr = reinterpret_cast<double2*>(base + 4 * mpad);
  double2* ff = reinterpret_cast<double2*>(base + 6 * mpad);
  double isq;
  tau_factor(N, sig, lam[m], e, h, bb, Q, &isq);
  const int Mp = (N - sig) / 2 + 1;
  for (int i = 0; i < Mp; ++i) rr[i] = r[(size_t)m * ny + 2 * i + sig];
  const double2 s = sig == 0 ? 0.5 * (top[m] + bot[m]) : 0.5 * (top[m] - bot[m]);
  tau_solve(N, sig, rr, ff, TabLocal{e, h, bb, Q}, isq, s);
  for (int i = 0; i < Mp; ++i) f[(size_t)m * ny + 2 * i + sig] = ff[i];
}

}  // namespace chdns

namespace {

// Device address of the scratch array, looked up once per device.
constexpr int kMaxDevices = 64;
double* g_noalloc_ptr[kMaxDevices] = {nullptr};
std::mutex g_noalloc_mu;

int noalloc_scratch(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CH_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_tau_noalloc_scratch) != cudaSuccess || !p) return CH_ERR_CUDA;
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return CH_OK;
}

}  // namespace

extern "C" int ch_tau_helmholtz_noalloc(int ny, int M, const double* d_lam, const double* d_r,
                                        const double* d_top, const double* d_bot, double* d_f, void* stream) {
  if (ny < 5 || ny > chdns::kMaxNy || M < 0) return CH_ERR_ARG;
  if (M == 0) return CH_OK;
  if (!d_lam || !d_r || !d_top || !d_bot || !d_f) return CH_ERR_ARG;
  const int mpad = ((ny / 2 + 1) + 1) & ~1;  // even, keeps the complex work vectors 16-byte aligned
  if ((size_t)2 * M * 8 * mpad > kNoAllocScratchDoubles) return CH_ERR_ARG;
  double* scratch = nullptr;
  const int rc = noalloc_scratch(&scratch);
  if (rc != CH_OK) return rc;
  const long n = 2L * M;
  chdns::tau_helmholtz_noalloc_kernel<<<(unsigned)((n + 63) / 64), 64, 0, static_cast<cudaStream_t>(stream)>>>(
      ny, M, mpad, d_lam, reinterpret_cast<const double2*>(d_r), reinterpret_cast<const double2*>(d_top),
      reinterpret_cast<const double2*>(d_bot), reinterpret_cast<double2*>(d_f), scratch);
  return cudaGetLastError() == cudaSuccess ? CH_OK : CH_ERR_CUDA;
}
