// Seeded O-grid meshes around a symmetric 4-digit airfoil (host code): the workload meshes
// standing in for the paper's NACA0012 mesh (Sec. 6.1), generated inside the library so that
// a caller needs no mesh of its own.  The construction, step by step:
//  - n_theta wall points counter-clockwise from the trailing edge, equally spaced in arc
//    length of the airfoil surface x = (1 + cos b)/2, y = +-t(x) (closed trailing edge,
//    thickness 12%), the arc length tabulated on 40001 equally spaced b in [0, 2 pi] and
//    inverted by linear interpolation; for even n_theta the leading edge b = pi exactly;
//  - far-field circle of radius r_far about (0.5, 0) at the same angles b;
//  - n_r + 1 rings by geometric stretching s_j = (q^j - 1)/(q^n_r - 1), q = 1 + 4/n_r;
//  - interior vertices moved by 0.1 h (u1, u2), h the distance to the nearest of the four
//    grid neighbours at that moment (rings 1 .. n_r - 1 in order, k inner), u1, u2 in [-1, 1)
//    the next two numbers of the counter-based SplitMix64 generator;
//  - each quad (k, j) split into two triangles, diagonal alternating with k + j, oriented
//    counter-clockwise; faces on ring 0 tagged wall (1), on ring n_r far field (2).
// The arithmetic follows the operation order of the package's input generator, so both
// produce the same mesh (connectivity exactly, coordinates to rounding of the libm calls).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "context.h"

namespace pp {
namespace {

uint64_t splitmix64(uint64_t seed, uint64_t counter) {
  uint64_t z = seed + (counter + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

double uniform_pm1(uint64_t seed, uint64_t counter) {
  return -1.0 + 2.0 * ((double)(splitmix64(seed, counter) >> 11) * (1.0 / 9007199254740992.0));
}

double half_thickness(double x, double t) {
  x = std::min(std::max(x, 0.0), 1.0);
  const double a = 0.2969 * std::sqrt(x);
  const double b = 0.1260 * x;
  const double c = 0.3516 * (x * x);
  const double d = 0.2843 * std::pow(x, 3.0);
  const double e = 0.1036 * std::pow(x, 4.0);
  return 5.0 * t * ((((a - b) - c) + d) - e);
}

}  // namespace

int ogrid_generate(int n_theta, int n_r, double r_far, uint64_t seed, std::vector<double>& verts,
                   std::vector<int32_t>& tris, std::vector<int32_t>& ftag) {
  if (n_theta < 3 || n_r < 1 || !(r_far > 1.0)) return PP_EINVAL;
  const double t = 0.12, jitter = 0.1;
  const double two_pi = 2.0 * M_PI;
  // arc length of the surface on the fine parametrization
  const int NF = 40001;
  std::vector<double> bf(NF), xf(NF), yf(NF), sf(NF);
  const double step = two_pi / (NF - 1);
  for (int i = 0; i < NF; ++i) bf[i] = (double)i * step + 0.0;
  bf[NF - 1] = two_pi;
  for (int i = 0; i < NF; ++i) {
    xf[i] = 0.5 * (1.0 + std::cos(bf[i]));
    yf[i] = half_thickness(xf[i], t) * (std::sin(bf[i]) >= 0.0 ? 1.0 : -1.0);
  }
  sf[0] = 0.0;
  for (int i = 1; i < NF; ++i) sf[i] = sf[i - 1] + std::hypot(xf[i] - xf[i - 1], yf[i] - yf[i - 1]);
  std::vector<double> beta(n_theta);
  for (int k = 0; k < n_theta; ++k) {
    const double x = sf[NF - 1] * (double)k / (double)n_theta;
    if (x >= sf[NF - 1]) {
      beta[k] = bf[NF - 1];
      continue;
    }
    const int j = (int)(std::upper_bound(sf.begin(), sf.end(), x) - sf.begin()) - 1;
    const double slope = (bf[j + 1] - bf[j]) / (sf[j + 1] - sf[j]);
    beta[k] = slope * (x - sf[j]) + bf[j];
  }
  if (n_theta % 2 == 0) beta[n_theta / 2] = M_PI;
  std::vector<double> wx(n_theta), wy(n_theta), fx(n_theta), fy(n_theta);
  for (int k = 0; k < n_theta; ++k) {
    const double sb = std::sin(beta[k]);
    wx[k] = 0.5 * (1.0 + std::cos(beta[k]));
    wy[k] = half_thickness(wx[k], t) * (sb >= 0.0 ? 1.0 : -1.0);
    if (std::fabs(sb) < 1e-14) wy[k] = 0.0;
    fx[k] = 0.5 + r_far * std::cos(beta[k]);
    fy[k] = r_far * sb;
  }
  const double q = 1.0 + 4.0 / n_r;
  std::vector<double> s(n_r + 1);
  const double qn = std::pow(q, (double)n_r) - 1.0;
  for (int j = 0; j <= n_r; ++j) s[j] = (std::pow(q, (double)j) - 1.0) / qn;
  const int nv = n_theta * (n_r + 1);
  verts.assign(2 * (size_t)nv, 0.0);
  auto X = [&](int k, int j) -> double& { return verts[2 * ((size_t)k * (n_r + 1) + j)]; };
  auto Y = [&](int k, int j) -> double& { return verts[2 * ((size_t)k * (n_r + 1) + j) + 1]; };
  for (int k = 0; k < n_theta; ++k)
    for (int j = 0; j <= n_r; ++j) {
      X(k, j) = wx[k] + s[j] * (fx[k] - wx[k]);
      Y(k, j) = wy[k] + s[j] * (fy[k] - wy[k]);
    }
  if (n_r >= 2) {
    uint64_t draw = 0;
    for (int j = 1; j < n_r; ++j)
      for (int k = 0; k < n_theta; ++k) {
        const double x0 = X(k, j), y0 = Y(k, j);
        const int kk[4] = {(k + 1) % n_theta, (k - 1 + n_theta) % n_theta, k, k};
        const int jj[4] = {j, j, j + 1, j - 1};
        double h = 0.0;
        for (int c = 0; c < 4; ++c) {
          const double dx = x0 - X(kk[c], jj[c]), dy = y0 - Y(kk[c], jj[c]);
          const double dd = dx * dx;
          const double d = std::sqrt(dd + dy * dy);
          if (c == 0 || d < h) h = d;
        }
        X(k, j) = x0 + jitter * h * uniform_pm1(seed, draw);
        Y(k, j) = y0 + jitter * h * uniform_pm1(seed, draw + 1);
        draw += 2;
      }
  }
  const int nt = 2 * n_theta * n_r;
  tris.assign(3 * (size_t)nt, 0);
  ftag.assign(3 * (size_t)nt, 0);
  auto vid = [&](int k, int j) { return k * (n_r + 1) + j; };
  int e = 0;
  for (int k = 0; k < n_theta; ++k) {
    const int k1 = (k + 1) % n_theta;
    for (int j = 0; j < n_r; ++j) {
      const int a = vid(k, j), b = vid(k1, j), c = vid(k1, j + 1), d = vid(k, j + 1);
      const int t0[3] = {a, b, (k + j) % 2 == 0 ? c : d};
      const int t1[3] = {(k + j) % 2 == 0 ? a : b, c, d};
      for (const int* tt : {t0, t1}) {
        int v0 = tt[0], v1 = tt[1], v2 = tt[2];
        const double ax = verts[2 * v0], ay = verts[2 * v0 + 1];
        const double area2 =
            (verts[2 * v1] - ax) * (verts[2 * v2 + 1] - ay) - (verts[2 * v1 + 1] - ay) * (verts[2 * v2] - ax);
        if (area2 < 0.0) std::swap(v1, v2);
        tris[3 * e] = v0;
        tris[3 * e + 1] = v1;
        tris[3 * e + 2] = v2;
        ++e;
      }
    }
  }
  for (int el = 0; el < nt; ++el)
    for (int f = 0; f < 3; ++f) {
      const int ra = tris[3 * el + f] % (n_r + 1), rb = tris[3 * el + (f + 1) % 3] % (n_r + 1);
      ftag[3 * el + f] = (ra == 0 && rb == 0) ? 1 : ((ra == n_r && rb == n_r) ? 2 : 0);
    }
  return PP_OK;
}

}  // namespace pp

extern "C" {

int pp_ogrid_generate(int n_theta, int n_r, double r_far, uint64_t seed, double* verts, int32_t* tris,
                      int32_t* ftag, int* nv, int* nt) {
  std::vector<double> v;
  std::vector<int32_t> t, g;
  const int st = pp::ogrid_generate(n_theta, n_r, r_far, seed, v, t, g);
  if (st != PP_OK) return st;
  if (nv) *nv = (int)(v.size() / 2);
  if (nt) *nt = (int)(t.size() / 3);
  if (verts) std::copy(v.begin(), v.end(), verts);
  if (tris) std::copy(t.begin(), t.end(), tris);
  if (ftag) std::copy(g.begin(), g.end(), ftag);
  return PP_OK;
}

int pp_mesh_ogrid(pp_ctx* ctx, int n_theta, int n_r, double r_far, uint64_t seed, pp_mesh** out) {
  if (!ctx || !out) return pp::set_error(ctx, PP_EINVAL, "pp_mesh_ogrid: null argument");
  std::vector<double> v;
  std::vector<int32_t> t, g;
  if (pp::ogrid_generate(n_theta, n_r, r_far, seed, v, t, g) != PP_OK)
    return pp::set_error(ctx, PP_EINVAL, "pp_mesh_ogrid: need n_theta >= 3, n_r >= 1, r_far > 1");
  return pp_mesh_create(ctx, v.data(), (int)(v.size() / 2), t.data(), g.data(), (int)(t.size() / 3), out);
}

}  // extern "C"
