// Host check of pf::local::reverse against central differences of
// pf::local::forward (double precision, random inputs in physical ranges):
// for random output adjoints a and input directions d,
//   <a, (F(x + h d) - F(x - h d)) / 2h>  ==  <reverse(x, a), d>.
// Also the three parameter directions.  Prints one line per trial:
//   trial rel_err_inputs rel_err_eps rel_err_Omega rel_err_sigma
#include <cstdio>
#include <random>

#include "../../paper_2407_01651_gb300/csrc/pf_local.cuh"

using namespace pf::local;
using R = double;

static const int NIN = 9 + 9 + 5 + 5 + 1 + 5 + 4 + 5;   // 43
static const int NOUT = 9 + 9 + 5 + 5 + 1 + 5 + 5;      // 39

static void pack_in(const In<R>& a, R* v) {
  int k = 0;
  for (int i = 0; i < 9; ++i) v[k++] = a.f[i];
  for (int i = 0; i < 9; ++i) v[k++] = a.h[i];
  for (int i = 0; i < 5; ++i) v[k++] = a.g[i];
  for (int i = 0; i < 5; ++i) v[k++] = a.s[i];
  v[k++] = a.psio;
  v[k++] = a.gpx; v[k++] = a.gpy; v[k++] = a.lphi; v[k++] = a.gsx; v[k++] = a.gsy;
  v[k++] = a.dvxx; v[k++] = a.dvxy; v[k++] = a.dvyx; v[k++] = a.dvyy;
  v[k++] = a.phio; v[k++] = a.Co; v[k++] = a.Qo; v[k++] = a.vxo; v[k++] = a.vyo;
}
static void unpack_in(const R* v, In<R>& a) {
  int k = 0;
  for (int i = 0; i < 9; ++i) a.f[i] = v[k++];
  for (int i = 0; i < 9; ++i) a.h[i] = v[k++];
  for (int i = 0; i < 5; ++i) a.g[i] = v[k++];
  for (int i = 0; i < 5; ++i) a.s[i] = v[k++];
  a.psio = v[k++];
  a.gpx = v[k++]; a.gpy = v[k++]; a.lphi = v[k++]; a.gsx = v[k++]; a.gsy = v[k++];
  a.dvxx = v[k++]; a.dvxy = v[k++]; a.dvyx = v[k++]; a.dvyy = v[k++];
  a.phio = v[k++]; a.Co = v[k++]; a.Qo = v[k++]; a.vxo = v[k++]; a.vyo = v[k++];
}
static void pack_out(const Out<R>& o, R* v) {
  int k = 0;
  for (int i = 0; i < 9; ++i) v[k++] = o.f[i];
  for (int i = 0; i < 9; ++i) v[k++] = o.h[i];
  for (int i = 0; i < 5; ++i) v[k++] = o.gpre[i];
  for (int i = 0; i < 5; ++i) v[k++] = o.gpost[i];
  v[k++] = o.rr;
  for (int i = 0; i < 5; ++i) v[k++] = o.s[i];
  v[k++] = o.phi; v[k++] = o.C; v[k++] = o.vx; v[k++] = o.vy; v[k++] = o.Q;
}
static void unpack_out(const R* v, Out<R>& o) {
  int k = 0;
  for (int i = 0; i < 9; ++i) o.f[i] = v[k++];
  for (int i = 0; i < 9; ++i) o.h[i] = v[k++];
  for (int i = 0; i < 5; ++i) o.gpre[i] = v[k++];
  for (int i = 0; i < 5; ++i) o.gpost[i] = v[k++];
  o.rr = v[k++];
  for (int i = 0; i < 5; ++i) o.s[i] = v[k++];
  o.phi = v[k++]; o.C = v[k++]; o.vx = v[k++]; o.vy = v[k++]; o.Q = v[k++];
  o.U = o.p = o.mu = 0;
}

static Coef<R> coef(R eps, R Omega, R sigma, double ang) {
  Coef<R> c{};
  const R rho_l = 1.0, rho_g = 0.1, nu = 0.1, W = 4.0, Mphi = 0.1, bphi = 0.25, bpsi = 0.25,
          bint = 0.75, W0 = 4.0, tau0 = 320.0, k = 0.15, D = 0.1, g = 1e-3;
  const R s_nu = 1.0 / (3 * nu + 0.5);
  c.rho_g = rho_g; c.drho = rho_l - rho_g; c.ge2 = 1e-6; c.gat2 = 1e-4;
  c.kappa = std::sqrt(2 * bphi) / W; c.fs_coef = 6 * sigma / (W * std::sqrt(2 * bphi));
  c.Wphi2 = W * W; c.M_phi = Mphi; c.two_bphi = 2 * bphi; c.two_bint = 2 * bint;
  c.four_bpsi = 4 * bpsi; c.lam = D * tau0 / ((47.0 / 75.0) * W0 * W0);
  c.Mcinf = 1 - (1 - k) * Omega; c.theta = -c.Mcinf * Omega / (1 - (1 - k) * Omega);
  c.inv_tau0 = 1 / tau0; c.c_s1 = 3 * W0 * W0 / tau0; c.W0 = W0;
  c.a_at = 1 / (2 * std::sqrt(2.0)); c.k = k; c.D = D; c.g = g;
  c.s_e = 1.0; c.s_eps = 1.0; c.s_q = 8 * (2 - s_nu) / (8 - s_nu); c.s_nu = s_nu;
  c.s_phi = 1 / (3 * Mphi + 0.5);
  c.eps = eps; c.ct = std::cos(ang); c.sn = std::sin(ang); c.rho_bar = 0.9;
  return c;
}

int main() {
  std::mt19937_64 rng(12345);
  std::uniform_real_distribution<R> U(-1, 1), P(0, 1);
  const R eps0 = 0.05, Om0 = 0.55, sig0 = 1e-3;
  int bad = 0;
  for (int trial = 0; trial < 200; ++trial) {
    const double ang = 1.5 * P(rng);
    In<R> in{};
    const R phi = 0.05 + 0.9 * P(rng), psi = -0.95 + 1.9 * P(rng), C = 0.1 + 0.9 * P(rng);
    const R w9[9] = {4. / 9, 1. / 9, 1. / 9, 1. / 9, 1. / 9, 1. / 36, 1. / 36, 1. / 36, 1. / 36};
    const R w5[5] = {1. / 3, 1. / 6, 1. / 6, 1. / 6, 1. / 6};
    for (int i = 0; i < 9; ++i) {
      in.f[i] = 1e-3 * U(rng);
      in.h[i] = w9[i] * phi * (1 + 0.05 * U(rng));
    }
    for (int i = 0; i < 5; ++i) {
      in.g[i] = w5[i] * psi + 0.01 * U(rng);
      in.s[i] = w5[i] * C * (1 + 0.05 * U(rng));
    }
    in.psio = psi + 0.01 * U(rng);
    in.gpx = 0.05 * U(rng); in.gpy = 0.05 * U(rng); in.lphi = 0.01 * U(rng);
    in.gsx = 0.1 * U(rng); in.gsy = 0.1 * U(rng);
    in.dvxx = 1e-3 * U(rng); in.dvxy = 1e-3 * U(rng); in.dvyx = 1e-3 * U(rng);
    in.dvyy = 1e-3 * U(rng);
    in.phio = phi + 0.01 * U(rng); in.Co = C + 0.01 * U(rng); in.Qo = 0.1 * U(rng);
    in.vxo = 1e-2 * U(rng); in.vyo = 1e-2 * U(rng);

    R a[NOUT], d[NIN], x[NIN];
    for (int k = 0; k < NOUT; ++k) a[k] = U(rng);
    for (int k = 0; k < NIN; ++k) d[k] = U(rng);
    pack_in(in, x);
    // scale directions to each input's size
    for (int k = 0; k < NIN; ++k) d[k] *= (std::fabs(x[k]) + 1e-3);

    Out<R> ao;
    unpack_out(a, ao);
    In<R> ai{};
    ParGrad<R> pg{0, 0, 0};
    const Coef<R> c0 = coef(eps0, Om0, sig0, ang);
    reverse(in, c0, c0.fs_coef / sig0, ao, ai, pg);
    R gi[NIN];
    pack_in(ai, gi);
    R adj = 0;
    for (int k = 0; k < NIN; ++k) adj += gi[k] * d[k];

    auto dot_out = [&](const In<R>& xin, const Coef<R>& c) {
      Out<R> o;
      forward(xin, c, o);
      R v[NOUT];
      pack_out(o, v);
      R s = 0;
      for (int k = 0; k < NOUT; ++k) s += a[k] * v[k];
      return s;
    };
    const R h = 1e-6;
    R xp[NIN], xm[NIN];
    for (int k = 0; k < NIN; ++k) { xp[k] = x[k] + h * d[k]; xm[k] = x[k] - h * d[k]; }
    In<R> ip{}, im{};
    unpack_in(xp, ip);
    unpack_in(xm, im);
    const R fd = (dot_out(ip, c0) - dot_out(im, c0)) / (2 * h);
    const R e_in = std::fabs(adj - fd) / (std::fabs(fd) + 1e-12);
    // parameters
    const R he = 1e-6 * eps0, ho = 1e-6 * Om0, hs = 1e-2 * sig0;  // sigma enters linearly via F_s
    const R fe = (dot_out(in, coef(eps0 + he, Om0, sig0, ang)) -
                  dot_out(in, coef(eps0 - he, Om0, sig0, ang))) / (2 * he);
    const R fo = (dot_out(in, coef(eps0, Om0 + ho, sig0, ang)) -
                  dot_out(in, coef(eps0, Om0 - ho, sig0, ang))) / (2 * ho);
    const R fs = (dot_out(in, coef(eps0, Om0, sig0 + hs, ang)) -
                  dot_out(in, coef(eps0, Om0, sig0 - hs, ang))) / (2 * hs);
    const R e_e = std::fabs(pg.eps - fe) / (std::fabs(fe) + 1e-10);
    const R e_o = std::fabs(pg.Omega - fo) / (std::fabs(fo) + 1e-10);
    const R e_s = std::fabs(pg.sigma - fs) / (std::fabs(fs) + 1e-10);
    std::printf("%d %.3e %.3e %.3e %.3e\n", trial, e_in, e_e, e_o, e_s);
    if (e_in > 1e-6 || e_e > 1e-5 || e_o > 1e-5 || e_s > 1e-5) ++bad;
  }
  std::printf("bad %d\n", bad);
  return bad ? 1 : 0;
}
