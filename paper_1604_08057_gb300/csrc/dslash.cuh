// Per-site Wilson-Dirac arithmetic (App. A, Eqs. WD_op and WD_G) with rank-2
// spin projection in the Euclidean chiral basis
//   gamma_k = [[0, -i sigma_k], [i sigma_k, 0]],  gamma_4 = [[0, 1], [1, 0]],
//   gamma5 = diag(1, 1, -1, -1).
// For psi = (u0, u1, d0, d1) (upper/lower spin pairs, each a colour vector),
// (1 +- gamma_nu) psi = (h, L h) with the half spinor h = P psi; only h is
// multiplied by the link, and L rebuilds the lower pair.
#pragma once
#include "common.cuh"

namespace ov {

template <typename R> struct Half { cplx<R> h[2][3]; };

// h = upper pair of (1 + sgn*gamma_nu) psi
template <int NU, int SGN, typename R>
OV_HD void spin_project(const Spinor<R>& p, Half<R>& o) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const cplx<R> u0 = p.c[0 * 3 + a], u1 = p.c[1 * 3 + a], d0 = p.c[2 * 3 + a], d1 = p.c[3 * 3 + a];
    if (NU == 0) {          // x: -/+ i sigma_1 d = -/+ i (d1, d0)
      o.h[0][a] = SGN > 0 ? u0 + times_mi(d1) : u0 + times_i(d1);
      o.h[1][a] = SGN > 0 ? u1 + times_mi(d0) : u1 + times_i(d0);
    } else if (NU == 1) {   // y: -/+ i sigma_2 d = -/+ (d1, -d0)
      o.h[0][a] = SGN > 0 ? u0 - d1 : u0 + d1;
      o.h[1][a] = SGN > 0 ? u1 + d0 : u1 - d0;
    } else if (NU == 2) {   // z: -/+ i sigma_3 d = -/+ i (d0, -d1)
      o.h[0][a] = SGN > 0 ? u0 + times_mi(d0) : u0 + times_i(d0);
      o.h[1][a] = SGN > 0 ? u1 + times_i(d1) : u1 + times_mi(d1);
    } else {                // t: u +/- d
      o.h[0][a] = SGN > 0 ? u0 + d0 : u0 - d0;
      o.h[1][a] = SGN > 0 ? u1 + d1 : u1 - d1;
    }
  }
}

// acc += s * (h, L h), the four spins of (1 + sgn*gamma_nu) psi rebuilt from h
template <int NU, int SGN, typename R>
OV_HD void spin_reconstruct_add(Spinor<R>& acc, const Half<R>& o, R s) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const cplx<R> h0 = o.h[0][a], h1 = o.h[1][a];
    cplx<R> l0, l1;
    if (NU == 0) {          // lower = +/- i sigma_1 h = +/- i (h1, h0)
      l0 = SGN > 0 ? times_i(h1) : times_mi(h1);
      l1 = SGN > 0 ? times_i(h0) : times_mi(h0);
    } else if (NU == 1) {   // lower = +/- i sigma_2 h = +/- (h1, -h0)
      l0 = SGN > 0 ? h1 : -h1;
      l1 = SGN > 0 ? -h0 : h0;
    } else if (NU == 2) {   // lower = +/- i sigma_3 h = +/- i (h0, -h1)
      l0 = SGN > 0 ? times_i(h0) : times_mi(h0);
      l1 = SGN > 0 ? times_mi(h1) : times_i(h1);
    } else {                // lower = +/- h
      l0 = SGN > 0 ? h0 : -h0;
      l1 = SGN > 0 ? h1 : -h1;
    }
    acc.c[0 * 3 + a] = acc.c[0 * 3 + a] + s * h0;
    acc.c[1 * 3 + a] = acc.c[1 * 3 + a] + s * h1;
    acc.c[2 * 3 + a] = acc.c[2 * 3 + a] + s * l0;
    acc.c[3 * 3 + a] = acc.c[3 * 3 + a] + s * l1;
  }
}

// o = U h (per spin of the half spinor)
template <typename R>
OV_HD void link_mul(const Mat3<R>& u, const Half<R>& h, Half<R>& o) {
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cplx<R> t = u.m[a * 3 + 0] * h.h[s][0];
      cmac(t, u.m[a * 3 + 1], h.h[s][1]);
      cmac(t, u.m[a * 3 + 2], h.h[s][2]);
      o.h[s][a] = t;
    }
}
// o = U^dagger h
template <typename R>
OV_HD void link_dag_mul(const Mat3<R>& u, const Half<R>& h, Half<R>& o) {
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cplx<R> t = conj(u.m[0 * 3 + a]) * h.h[s][0];
      cmac(t, conj(u.m[1 * 3 + a]), h.h[s][1]);
      cmac(t, conj(u.m[2 * 3 + a]), h.h[s][2]);
      o.h[s][a] = t;
    }
}

// Loader of a single field: psi(s)
template <typename R>
struct FieldLoad {
  const R* f;
  int64_t V;
  OV_HD void operator()(int64_t s, Spinor<R>& o) const { load_spinor_ro(f, V, s, o); }
};

// One direction's two hops of sum_nu [f (1+g) U_nu(x) psi(x+nu) + f^-1 (1-g) U_nu(x-nu)^dag psi(x-nu)]
// `ld(s, spinor)` supplies psi at any site (a field or a combination of fields).
template <int NU, typename R, typename LD>
OV_HD void hop_dir(Spinor<R>& acc, const LD& ld, const R* u, const Geom& g, int64_t s, const int c[4],
                   R ft, R ftinv) {
  const R ff = (NU == 3) ? ft : R(1);
  const R fb = (NU == 3) ? ftinv : R(1);
  Spinor<R> nb;
  Half<R> h, uh;
  Mat3<R> lk;
  const int64_t sf = neighbour(g, s, c, NU, +1);
  ld(sf, nb);
  spin_project<NU, +1>(nb, h);
  load_link(u, g.V, s, NU, lk);
  link_mul(lk, h, uh);
  spin_reconstruct_add<NU, +1>(acc, uh, ff);
  const int64_t sb = neighbour(g, s, c, NU, -1);
  ld(sb, nb);
  spin_project<NU, -1>(nb, h);
  load_link(u, g.V, sb, NU, lk);
  link_dag_mul(lk, h, uh);
  spin_reconstruct_add<NU, -1>(acc, uh, fb);
}

// out(x) = gamma5 D_w psi (x), with ft = e^{mu_eff} on forward temporal hops.
// H = gamma5 D_w(mu) uses mu_eff = mu; H^dagger = gamma5 D_w(-mu) uses -mu.
template <typename R, typename LD>
OV_HD void h_site_ld(const LD& ld, const R* u, const Geom& g, int64_t s, R kappa, R ft, R ftinv,
                     Spinor<R>& out) {
  int c[4];
  site_coords(g, s, c);
  Spinor<R> acc;
  spinor_zero(acc);
  hop_dir<0>(acc, ld, u, g, s, c, ft, ftinv);
  hop_dir<1>(acc, ld, u, g, s, c, ft, ftinv);
  hop_dir<2>(acc, ld, u, g, s, c, ft, ftinv);
  hop_dir<3>(acc, ld, u, g, s, c, ft, ftinv);
  Spinor<R> p;
  ld(s, p);
#pragma unroll
  for (int i = 0; i < 6; ++i) out.c[i] = p.c[i] - kappa * acc.c[i];
#pragma unroll
  for (int i = 6; i < 12; ++i) out.c[i] = kappa * acc.c[i] - p.c[i];
}

template <typename R>
OV_HD void h_site(const R* f, const R* u, const Geom& g, int64_t s, R kappa, R ft, R ftinv,
                  Spinor<R>& out) {
  FieldLoad<R> ld{f, g.V};
  h_site_ld(ld, u, g, s, kappa, ft, ftinv, out);
}

// NS right-hand sides sharing every link load: out[i] = gamma5 D_w psi_i with
// ft[i] = e^{mu_i} on forward temporal hops (H uses mu, H^dagger uses -mu).
template <int NU, int NS, typename R, typename LD>
OV_HD void hop_dir_multi(Spinor<R> (&acc)[NS], const LD (&ld)[NS], const R* u, const Geom& g, int64_t s,
                         const int c[4], const R (&ft)[NS], const R (&fti)[NS]) {
  Spinor<R> nb;
  Half<R> h, uh;
  Mat3<R> lk;
  const int64_t sf = neighbour(g, s, c, NU, +1);
  load_link(u, g.V, s, NU, lk);
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    ld[i](sf, nb);
    spin_project<NU, +1>(nb, h);
    link_mul(lk, h, uh);
    spin_reconstruct_add<NU, +1>(acc[i], uh, NU == 3 ? ft[i] : R(1));
  }
  const int64_t sb = neighbour(g, s, c, NU, -1);
  load_link(u, g.V, sb, NU, lk);
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    ld[i](sb, nb);
    spin_project<NU, -1>(nb, h);
    link_dag_mul(lk, h, uh);
    spin_reconstruct_add<NU, -1>(acc[i], uh, NU == 3 ? fti[i] : R(1));
  }
}

template <int NS, typename R, typename LD>
OV_HD void h_site_multi(const LD (&ld)[NS], const R* u, const Geom& g, int64_t s, R kappa, const R (&ft)[NS],
                        const R (&fti)[NS], Spinor<R> (&out)[NS]) {
  int c[4];
  site_coords(g, s, c);
#pragma unroll
  for (int i = 0; i < NS; ++i) spinor_zero(out[i]);
  hop_dir_multi<0>(out, ld, u, g, s, c, ft, fti);
  hop_dir_multi<1>(out, ld, u, g, s, c, ft, fti);
  hop_dir_multi<2>(out, ld, u, g, s, c, ft, fti);
  hop_dir_multi<3>(out, ld, u, g, s, c, ft, fti);
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    Spinor<R> p;
    ld[i](s, p);
#pragma unroll
    for (int q = 0; q < 6; ++q) out[i].c[q] = p.c[q] - kappa * out[i].c[q];
#pragma unroll
    for (int q = 6; q < 12; ++q) out[i].c[q] = kappa * out[i].c[q] - p.c[q];
  }
}

// Link-gradient contribution of one rank-one term a b^dagger for direction NU,
// on half spinors.  With h = P_+(b(x+nu)) the upper pair of (1+gamma_nu) b(x+nu),
//   sum_s a(x)_s conj((gamma5 (1+gamma_nu) b(x+nu))_s) = sum_t a~_t conj(h_t),
// where a~ = P_-(a(x)) (the lower pair enters through gamma5 and the adjoint
// of the reconstruction); likewise for the backward hop with the signs swapped:
//   forward:  G[c][d] += cf * sum_t a~_t[c] conj(h_t[d]),   a~ = P_-(a(x)),   h = P_+(b(x+nu))
//   backward: G[c][d] += cb * sum_t conj(a'_t[d]) h'_t[c],  a' = P_+(a(x+nu)), h' = P_-(b(x))
// (cf = -kappa f_nu, cb = -kappa / f_nu).  Gd collects forward minus backward.
template <int NU, typename R>
OV_HD void force_half_fwd(const Spinor<R>& ax, const Spinor<R>& bxf, R cf, cplx<R> (&G)[9], cplx<R> (&Gd)[9],
                          bool with_d) {
  Half<R> at, h;
  spin_project<NU, -1>(ax, at);
  spin_project<NU, +1>(bxf, h);
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      cplx<R> t = czero<R>();
      cdotac(t, h.h[0][d], at.h[0][c]);   // conj(h) * a~
      cdotac(t, h.h[1][d], at.h[1][c]);
      G[c * 3 + d] = G[c * 3 + d] + cf * t;
      if (with_d) Gd[c * 3 + d] = Gd[c * 3 + d] + cf * t;
    }
}
template <int NU, typename R>
OV_HD void force_half_bwd(const Spinor<R>& axf, const Spinor<R>& bx, R cb, cplx<R> (&G)[9], cplx<R> (&Gd)[9],
                          bool with_d) {
  Half<R> at, h;
  spin_project<NU, +1>(axf, at);
  spin_project<NU, -1>(bx, h);
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      cplx<R> t = czero<R>();
      cdotac(t, at.h[0][d], h.h[0][c]);   // conj(a') * h'
      cdotac(t, at.h[1][d], h.h[1][c]);
      G[c * 3 + d] = G[c * 3 + d] + cb * t;
      if (with_d) Gd[c * 3 + d] = Gd[c * 3 + d] - cb * t;
    }
}
template <int NU, typename R>
OV_HD void force_half(const Spinor<R>& ax, const Spinor<R>& bxf, const Spinor<R>& axf, const Spinor<R>& bx,
                      R cf, R cb, cplx<R> (&G)[9], cplx<R> (&Gd)[9], bool with_d) {
  force_half_fwd<NU>(ax, bxf, cf, G, Gd, with_d);
  force_half_bwd<NU>(axf, bx, cb, G, Gd, with_d);
}

// Loader of one half of a block field: psi(off + s) in a field of Vf sites
template <typename R>
struct FieldLoadOff {
  const R* f;
  int64_t Vf, off;
  OV_HD void operator()(int64_t s, Spinor<R>& o) const { load_spinor_ro(f, Vf, off + s, o); }
};

// Directional derivative of H along links E (ue, may be null) and mu (m):
//   dH psi = gamma5 [ -kappa sum_nu (f_nu (1+g_nu) E_nu(x) psi(x+nu) + f_nu^-1 (1-g_nu) E_nu(x-nu)^dag psi(x-nu))
//                     - kappa m (ft (1+g_4) U_4(x) psi(x+t) - ftinv (1-g_4) U_4(x-t)^dag psi(x-t)) ]
// (Eq. WD_op is affine in the links).  (dH)^dagger is the same with ft and ftinv
// exchanged and m -> -m.
template <typename R, typename LD>
OV_HD void dh_site_ld(const LD& ld, const R* ue, const R* u, const Geom& g, int64_t s, R kappa, R ft, R ftinv,
                      R m, Spinor<R>& out) {
  int c[4];
  site_coords(g, s, c);
  Spinor<R> acc;
  spinor_zero(acc);
  if (ue) {
    hop_dir<0>(acc, ld, ue, g, s, c, ft, ftinv);
    hop_dir<1>(acc, ld, ue, g, s, c, ft, ftinv);
    hop_dir<2>(acc, ld, ue, g, s, c, ft, ftinv);
    hop_dir<3>(acc, ld, ue, g, s, c, ft, ftinv);
  }
  if (m != R(0)) {
    Spinor<R> nb;
    Half<R> h, uh;
    Mat3<R> lk;
    const int64_t sf = neighbour(g, s, c, 3, +1);
    ld(sf, nb);
    spin_project<3, +1>(nb, h);
    load_link(u, g.V, s, 3, lk);
    link_mul(lk, h, uh);
    spin_reconstruct_add<3, +1>(acc, uh, m * ft);
    const int64_t sb = neighbour(g, s, c, 3, -1);
    ld(sb, nb);
    spin_project<3, -1>(nb, h);
    load_link(u, g.V, sb, 3, lk);
    link_dag_mul(lk, h, uh);
    spin_reconstruct_add<3, -1>(acc, uh, -m * ftinv);
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) out.c[i] = -kappa * acc.c[i];
#pragma unroll
  for (int i = 6; i < 12; ++i) out.c[i] = kappa * acc.c[i];
}

// gamma5 (1 + sgn*gamma_nu) b, all four spins (used by the force contraction)
template <int NU, int SGN, typename R>
OV_HD void g5_proj_full(const Spinor<R>& b, Spinor<R>& o) {
  Half<R> h;
  spin_project<NU, SGN>(b, h);
  spinor_zero(o);
  spin_reconstruct_add<NU, SGN>(o, h, R(1));
#pragma unroll
  for (int i = 6; i < 12; ++i) o.c[i] = -o.c[i];
}

}  // namespace ov
