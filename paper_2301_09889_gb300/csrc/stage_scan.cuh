// The no-slip implicit solves of one (mode, class, component, equation) spread
// over a group of four lanes, for handles with too few modes to fill the GPU
// with one thread per system (one environment of 120 to 8000 modes).
//
// Lane q of the group holds the block of coefficient indices
//   i = MH - 1 - q K - k,  k = 0 .. K - 1,  K = ceil(MH / 4),
// so lane 0 holds the top of the spectrum and lane 3 the bottom.  Every
// sequential sweep of the single-thread solve becomes a block sweep plus a
// combination across the four lanes:
//   - sums (wall rows, influence and flux sums): block sums, then a fixed
//     butterfly over the group;
//   - running sums from the top (the derivative walk of v): block prefix sums
//     plus the inclusive prefix of the block totals of the lanes above;
//   - the first-order recurrences of the tau elimination, a_j = alpha_j -
//     h_j a_{j+1} (downwards) and P_i = b_i P_{i-1} + a_i (upwards): each
//     block composes its affine maps, a Kogge-Stone scan composes the maps of
//     the lanes before it, and the block is swept again from its true input.
// The chains a thread waits on are K long instead of MH; the price is about
// half again the FP64 operations of the sweeps, which the under-filled FP64
// pipe of these handles absorbs.  Sums are formed in another order than the
// single-thread form, so the two forms agree to rounding, not bitwise.
#pragma once

#include "common.cuh"

namespace chdns {

namespace scan4 {

// the four lanes of this thread's group (groups of a warp may take different
// paths: every shuffle names only its own group)
__device__ __forceinline__ unsigned group_mask() { return 0xfu << (threadIdx.x & 28u); }

// sum over the four lanes of the group, the same bits on every lane
__device__ __forceinline__ double lane_sum(double x) {
  const unsigned m = group_mask();
  x = x + __shfl_xor_sync(m, x, 1, 4);
  return x + __shfl_xor_sync(m, x, 2, 4);
}

// exclusive prefix over lanes 0 .. q - 1 of a per-lane total
template <typename T>
__device__ __forceinline__ T lanes_above(T tot, int q) {
  const unsigned m = group_mask();
  T inc = tot;
#pragma unroll
  for (int o = 1; o < 4; o <<= 1) {
    const T v = __shfl_up_sync(m, inc, o, 4);
    if (q >= o) inc = inc + v;
  }
  const T ex = __shfl_up_sync(m, inc, 1, 4);
  return q == 0 ? (T)0 : ex;
}

// The input of lane q's block for a chain x -> A + B x composed block by
// block: downwards (lane 0 first, down = true) or upwards (lane 3 first); the
// first block's input is 0.
__device__ __forceinline__ double chain_input(double A, double B, int q, bool down) {
  const unsigned m = group_mask();
#pragma unroll
  for (int o = 1; o < 4; o <<= 1) {
    const double Ap = down ? __shfl_up_sync(m, A, o, 4) : __shfl_down_sync(m, A, o, 4);
    const double Bp = down ? __shfl_up_sync(m, B, o, 4) : __shfl_down_sync(m, B, o, 4);
    if (down ? q >= o : q + o <= 3) {
      A = fma_rn(B, Ap, A);  // (A, B) after (Ap, Bp)
      B = mul_rn(B, Bp);
    }
  }
  const double in = down ? __shfl_up_sync(m, A, 1, 4) : __shfl_down_sync(m, A, 1, 4);
  return (down ? q == 0 : q == 3) ? 0.0 : in;
}

}  // namespace scan4

template <int MH>
struct Blk {
  static constexpr int K = (MH + 3) / 4;
  __device__ static constexpr int i_of(int q, int k) { return MH - 1 - q * K - k; }
};

// Chebyshev-tau Dirichlet solve (tau_seq's rows) over a four-lane group.  On
// entry f[k] holds r at i = i_of(q, k) (0 outside 0 .. M - 1); on return the
// solution f_i, with the wall row sum_i f_i = wall.
template <int MH, class Tab>
__device__ __forceinline__ void tau_scan(int N, int ny, int sig, double (&f)[Blk<MH>::K], const Tab& T, double isq,
                                         double wall, const double* __restrict__ rowc, int q) {
  constexpr int K = Blk<MH>::K;
  const int M = (N - sig) / 2 + 1;
  // neighbours across the block edges: r at hi + 1 (bottom of the lane above)
  // and at lo - 1 (top of the lane below)
  const unsigned m = scan4::group_mask();
  const double above = __shfl_up_sync(m, f[K - 1], 1, 4), below = __shfl_down_sync(m, f[0], 1, 4);
  const double r_above = q == 0 ? 0.0 : above;
  const double r_below = q == 3 ? 0.0 : below;
  // alpha_j = e_j R_j in place (r_{j+1} kept from the previous step), and the
  // block's map a_bottom = A + B a_in
  double A = 0.0, B = 1.0;
  double r_up = r_above;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int j = Blk<MH>::i_of(q, k);
    const double rj = f[k];
    const double rlo = k + 1 < K ? f[k + 1] : r_below;
    if (j >= 1 && j < M) {
      const int n = 2 * j + sig;
      double R = fma_rn(-rowc[ny + n], rj, mul_rn(rowc[n], rlo));
      if (j + 1 < M) R = fma_rn(rowc[2 * ny + n], r_up, R);
      const double al = mul_rn(T.e(j), R);
      const double be = -T.h(j);
      f[k] = al;
      A = fma_rn(be, A, al);
      B = mul_rn(be, B);
    }
    r_up = rj;
  }
  double a = scan4::chain_input(A, B, q, true);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int j = Blk<MH>::i_of(q, k);
    if (j >= 1 && j < M) {
      a = fma_rn(-T.h(j), a, f[k]);
      f[k] = a;
    }
  }
  // upwards: P_i = b_i P_{i-1} + a_i from P_0 = 0; the block map and then the sweep
  A = 0.0;
  B = 1.0;
#pragma unroll
  for (int k = K - 1; k >= 0; --k) {
    const int i = Blk<MH>::i_of(q, k);
    if (i >= 1 && i < M) {
      A = fma_rn(T.b(i), A, f[k]);
      B = mul_rn(T.b(i), B);
    }
  }
  double Pp = scan4::chain_input(A, B, q, false);
  double s = 0.0;
#pragma unroll
  for (int k = K - 1; k >= 0; --k) {
    const int i = Blk<MH>::i_of(q, k);
    if (i >= 1 && i < M) {
      Pp = fma_rn(T.b(i), Pp, f[k]);
      f[k] = Pp;
      s += Pp;
    }
  }
  const double f0 = mul_rn(isq, wall - scan4::lane_sum(s));
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int i = Blk<MH>::i_of(q, k);
    if (i == 0) f[k] = f0;
    else if (i >= 1 && i < M) f[k] = fma_rn(T.Q(i), f0, f[k]);
  }
}

// omega_y of parity sq (omega_solve over a four-lane group)
template <int MH, typename RN, class GV, class HV, class Tab>
__device__ __forceinline__ void omega_scan(int N, int ny, int ppc, int sq, const GV& Gc, const HV& HGc,
                                           const typename cpx<RN>::T* Hx, const typename cpx<RN>::T* Hz, int r,
                                           double sgn, double kx, double kz, double cc, const StageCoef& sc,
                                           const Tab& T, double isq, const double* __restrict__ rowc, int q) {
  using CN = typename cpx<RN>::T;
  constexpr int K = Blk<MH>::K;
  const int ra = 1 - r;
  auto comp = [](const CN z, int qd) { return qd == 0 ? z.x : z.y; };
  const RN sgnn = (RN)sgn, kxn = (RN)kx, kzn = (RN)kz;
  const RN dtn = (RN)sc.dt, gan = (RN)sc.gamma, zen = (RN)sc.zeta;
  const int M = (N - sq) / 2 + 1;
  double f[K];
  double sum = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int i = Blk<MH>::i_of(q, k);
    f[k] = 0.0;
    if (i >= 0 && i < M) {
      const int n = 2 * i + sq;
      const double gn = Gc[n];
      const RN hg = mul_rn(sgnn, fma_rn(-kxn, comp(Hz[n * ppc], ra), mul_rn(kzn, comp(Hx[n * ppc], ra))));
      const RN hp = HGc[n];
      HGc[n] = hg;
      const RN qv = mul_rn(dtn, fma_rn(gan, hg, mul_rn(zen, hp)));
      f[k] = fma_rn(1.0 + cc, gn, (double)qv);
      sum += gn;
    }
  }
  tau_scan<MH>(N, ny, sq, f, T, isq, mul_rn(cc, scan4::lane_sum(sum)), rowc, q);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int i = Blk<MH>::i_of(q, k);
    if (i >= 0 && i < M) {
      const int n = 2 * i + sq;
      Gc[n] = fma_rn(-cc, Gc[n], f[k]);
    }
  }
}

// v of parity sv (v_solve over a four-lane group): the derivative walk as
// running sums from the top, the phi solve, the Poisson solve and the
// influence correction
template <int MH, typename RN, class VV, class HV, class Tab, class TabP>
__device__ __forceinline__ void v_scan(int N, int ny, int ppc, int sv, const VV& Vc, const HV& HVc,
                                       const typename cpx<RN>::T* Hx, const typename cpx<RN>::T* Hy,
                                       const typename cpx<RN>::T* Hz, int r, double sgn, double kx, double kz,
                                       double k2, double cc, const StageCoef& sc, const Tab& Th, double isq_h,
                                       const TabP& Tp, double isq_p, const double* vh, int vhs, double idv,
                                       double vw, const double* __restrict__ rowc, int q) {
  using CN = typename cpx<RN>::T;
  constexpr int K = Blk<MH>::K;
  const int ra = 1 - r;
  auto comp = [](const CN z, int qd) { return qd == 0 ? z.x : z.y; };
  const double dsv = 2.0 * sv;
  const RN dsvn = (RN)(2 * sv);
  const RN sgnn = (RN)sgn, kxn = (RN)kx, kzn = (RN)kz, k2n = (RN)k2;
  const RN dtn = (RN)sc.dt, gan = (RN)sc.gamma, zen = (RN)sc.zeta;
  const int M = (N - sv) / 2 + 1;
  double f[K];
  RN tk[K];
  // Dv: running sum from the top of 2 (no + 1) v_{no+1}, no = n + 1
  double dv = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int i = Blk<MH>::i_of(q, k);
    const int no = 2 * i + sv + 1;
    f[k] = 0.0;
    tk[k] = (RN)0;
    if (i >= 0 && i < M && no <= N) {
      const double vn1 = (no + 1 <= N) ? Vc[no + 1] : 0.0;
      dv = fma_rn((double)(4 * i + 4) + dsv, vn1, dv);
      tk[k] = mul_rn(sgnn, fma_rn(kxn, comp(Hx[no * ppc], ra), mul_rn(kzn, comp(Hz[no * ppc], ra))));
    }
    f[k] = dv;
  }
  const double dv_off = scan4::lanes_above(dv, q);
#pragma unroll
  for (int k = 0; k < K; ++k) f[k] = f[k] + dv_off;
  // D^2 v and Dt: running sums from the top of 2 (n + 1) Dv and 2 (n + 1) t
  double d2v = 0.0;
  RN dtt = (RN)0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int i = Blk<MH>::i_of(q, k);
    const int n = 2 * i + sv;
    if (i >= 0 && i < M) {
      d2v = fma_rn((double)(4 * i + 2) + dsv, f[k], d2v);
      dtt = fma_rn((RN)(4 * i + 2) + dsvn, (n + 1 <= N) ? tk[k] : (RN)0, dtt);
    }
    f[k] = d2v;
    tk[k] = dtt;
  }
  const double d2_off = scan4::lanes_above(d2v, q);
  const RN dt_off = scan4::lanes_above(dtt, q);
  // right-hand sides of the phi solve, and the wall sums of the old field
  double S0 = 0.0, S2 = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int i = Blk<MH>::i_of(q, k);
    const int n = 2 * i + sv;
    double rhs = 0.0;
    if (i >= 0 && i < M) {
      double d2 = f[k] + d2_off;
      RN dt2 = tk[k] + dt_off;
      if (n == 0) {
        d2 = 0.5 * d2;
        dt2 = (RN)0.5 * dt2;
      }
      const double vn = Vc[n];
      S0 += vn;
      S2 = fma_rn((double)n * n, vn, S2);
      const double phi = fma_rn(-k2, vn, d2);
      const RN hv = fma_rn(-k2n, comp(Hy[n * ppc], r), -dt2);
      const RN hp = HVc[n];
      HVc[n] = hv;
      const RN qv = mul_rn(dtn, fma_rn(gan, hv, mul_rn(zen, hp)));
      rhs = fma_rn(1.0 + cc, phi, (double)qv);
    }
    f[k] = rhs;
  }
  S0 = scan4::lane_sum(S0);
  S2 = scan4::lane_sum(S2);
  tau_scan<MH>(N, ny, sv, f, Th, isq_h, 0.0, rowc, q);
  const double s = fma_rn(cc, S0, ((sv == 0) ? 0.5 : -0.5) * vw);
  tau_scan<MH>(N, ny, sv, f, Tp, isq_p, s, rowc, q);
  double dp = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int i = Blk<MH>::i_of(q, k);
    if (i >= 0 && i < M) {
      const double n = 2 * i + sv;
      dp = fma_rn(n * n, f[k], dp);
    }
  }
  const double cI = mul_rn(fma_rn(cc, S2, -scan4::lane_sum(dp)), idv);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int i = Blk<MH>::i_of(q, k);
    if (i >= 0 && i < M) {
      const int n = 2 * i + sv;
      Vc[n] = fma_rn(-cc, Vc[n], fma_rn(cI, vh[i * vhs], f[k]));
    }
  }
}

// mean flow of parity s over a four-lane group (mean_solve)
template <int MH, typename RN, class Tab>
__device__ __forceinline__ void mean_scan(int N, int ny, int ppc, int s, int e, double* X, double* XP,
                                          const typename cpx<RN>::T* Hm, double cc, const StageCoef& sc,
                                          const Tab& T, double isq, const double* __restrict__ rowc,
                                          const double* __restrict__ u1, double u1_iflux, int q) {
  constexpr int K = Blk<MH>::K;
  const int M = (N - s) / 2 + 1;
  double f[K];
  double sum = 0.0, flux_old = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int i = Blk<MH>::i_of(q, k);
    f[k] = 0.0;
    if (i >= 0 && i < M) {
      const int n = 2 * i + s;
      const double xn = X[n];
      const double hv = (double)Hm[n * ppc].x;
      const double hp = XP[n];
      XP[n] = hv;
      sum += xn;
      if (s == 0) flux_old = fma_rn(2.0 / (1.0 - (double)n * n), xn, flux_old);
      f[k] = fma_rn(1.0 + cc, xn, mul_rn(sc.dt, fma_rn(sc.gamma, hv, mul_rn(sc.zeta, hp))));
    }
  }
  flux_old = scan4::lane_sum(flux_old);
  tau_scan<MH>(N, ny, s, f, T, isq, mul_rn(cc, scan4::lane_sum(sum)), rowc, q);
  double fc = 0.0;
  if (e == 0 && s == 0) {
    double flux = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int i = Blk<MH>::i_of(q, k);
      if (i >= 0 && i < M) flux = fma_rn(2.0 / (1.0 - 4.0 * (double)i * i), f[k], flux);
    }
    fc = mul_rn(fma_rn(cc, flux_old, sc.flux) - scan4::lane_sum(flux), u1_iflux);
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int i = Blk<MH>::i_of(q, k);
    if (i >= 0 && i < M) {
      const int n = 2 * i + s;
      double v = fma_rn(-cc, X[n], f[k]);
      if (e == 0 && s == 0) v = fma_rn(fc, u1[i], v);
      X[n] = v;
    }
  }
}

}  // namespace chdns
