// Floquet multipliers of a periodic orbit (Sec. 3.3, Eq. stab-def): the orbit is stable when
// every eigenvalue of Phi = du^(Nt)/du0 at the periodic u0 has modulus below one.  Phi is
// applied matrix-free by tangent sweeps (Eq. dirk-sens-mvp) over the stored linearization;
// an Arnoldi process of m steps with full classical Gram-Schmidt reorthogonalization builds
// the (m+1) x m Hessenberg matrix of Phi on the Krylov space, whose m x m leading block's
// eigenvalues (Ritz values) approximate the largest-modulus multipliers first.
//
// The Ritz values come from the Francis double-shift QR iteration on the Hessenberg block
// (host code, written from the textbook statement of the algorithm: implicit double-shift
// steps chasing a 3 x 3 bulge with Householder reflectors, deflation on negligible
// subdiagonal entries, 1 x 1 and 2 x 2 diagonal blocks read off at the end).
#include <algorithm>
#include <cmath>
#include <vector>

#include "context.h"
#include "../../include/pp_prof.h"

namespace pp {
namespace {

// eigenvalues of the 2 x 2 block [[a, b], [c, d]]
void eig2(double a, double b, double c, double d, double& r1, double& i1, double& r2, double& i2) {
  const double p = 0.5 * (a - d);
  const double q = p * p + b * c;
  const double m = 0.5 * (a + d);
  if (q >= 0.0) {
    const double s = std::sqrt(q);
    // the root of larger modulus first, the other from the determinant (no cancellation)
    const double big = m + (m >= 0.0 ? s : -s);
    const double det = a * d - b * c;
    r1 = big;
    r2 = big != 0.0 ? det / big : m - (m >= 0.0 ? s : -s);
    i1 = i2 = 0.0;
  } else {
    const double s = std::sqrt(-q);
    r1 = r2 = m;
    i1 = s;
    i2 = -s;
  }
}

// Householder reflector P = I - 2 v v^T / (v^T v) with P x = -sign(x0)|x| e1, for a
// vector of length 2 or 3; returns false if x is zero
bool house(int len, const double* x, double v[3]) {
  double nrm = 0.0;
  for (int i = 0; i < len; ++i) nrm += x[i] * x[i];
  nrm = std::sqrt(nrm);
  if (nrm == 0.0) return false;
  const double alpha = x[0] >= 0.0 ? nrm : -nrm;
  v[0] = x[0] + alpha;
  for (int i = 1; i < len; ++i) v[i] = x[i];
  if (len < 3) v[2] = 0.0;
  return true;
}

}  // namespace

// All eigenvalues of the n x n upper Hessenberg matrix H (row-major, leading dimension ld;
// overwritten).  Returns 0, or -1 if an eigenvalue did not converge in 60 n iterations.
int hessenberg_eigvals(int n, double* H, int ld, double* wr, double* wi) {
  auto h = [&](int i, int j) -> double& { return H[(size_t)i * ld + j]; };
  const double eps = 2.220446049250313e-16;
  int hi = n - 1;
  int iter = 0, total = 0;
  while (hi >= 0) {
    if (total > 60 * std::max(n, 1)) return -1;
    // deflation: the lowest l with a negligible subdiagonal entry above the active block
    int l = hi;
    while (l > 0) {
      const double s = std::fabs(h(l - 1, l - 1)) + std::fabs(h(l, l));
      if (std::fabs(h(l, l - 1)) <= eps * (s > 0.0 ? s : 1.0)) {
        h(l, l - 1) = 0.0;
        break;
      }
      --l;
    }
    if (l == hi) {  // 1 x 1 block
      wr[hi] = h(hi, hi);
      wi[hi] = 0.0;
      --hi;
      iter = 0;
      continue;
    }
    if (l == hi - 1) {  // 2 x 2 block
      eig2(h(hi - 1, hi - 1), h(hi - 1, hi), h(hi, hi - 1), h(hi, hi), wr[hi - 1], wi[hi - 1], wr[hi], wi[hi]);
      hi -= 2;
      iter = 0;
      continue;
    }
    ++iter;
    ++total;
    // shifts: the trailing 2 x 2 block's eigenvalues (sum s, product t); exceptional shifts
    // every tenth iteration without deflation
    double s, t;
    if (iter % 10 == 0) {
      const double e = std::fabs(h(hi, hi - 1)) + std::fabs(h(hi - 1, hi - 2));
      s = 1.5 * e + h(hi, hi);
      t = e * e;
    } else {
      s = h(hi - 1, hi - 1) + h(hi, hi);
      t = h(hi - 1, hi - 1) * h(hi, hi) - h(hi - 1, hi) * h(hi, hi - 1);
    }
    // first column of (H - s1)(H - s2) restricted to the active block
    double x[3];
    x[0] = h(l, l) * h(l, l) + h(l, l + 1) * h(l + 1, l) - s * h(l, l) + t;
    x[1] = h(l + 1, l) * (h(l, l) + h(l + 1, l + 1) - s);
    x[2] = h(l + 1, l) * h(l + 2, l + 1);
    for (int k = l; k <= hi - 2; ++k) {
      double v[3];
      if (house(3, x, v)) {
        const double vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        // rows k..k+2 from the left, columns from max(l, k-1) to hi
        for (int j = std::max(l, k - 1); j <= hi; ++j) {
          const double d = 2.0 * (v[0] * h(k, j) + v[1] * h(k + 1, j) + v[2] * h(k + 2, j)) / vv;
          h(k, j) -= d * v[0];
          h(k + 1, j) -= d * v[1];
          h(k + 2, j) -= d * v[2];
        }
        // columns k..k+2 from the right, rows l to min(k+3, hi)
        for (int i = l; i <= std::min(k + 3, hi); ++i) {
          const double d = 2.0 * (h(i, k) * v[0] + h(i, k + 1) * v[1] + h(i, k + 2) * v[2]) / vv;
          h(i, k) -= d * v[0];
          h(i, k + 1) -= d * v[1];
          h(i, k + 2) -= d * v[2];
        }
      }
      x[0] = h(k + 1, k);
      x[1] = h(k + 2, k);
      if (k < hi - 2) x[2] = h(k + 3, k);
    }
    // the last reflector is 2 x 2, on rows / columns hi-1 .. hi
    double v[3];
    if (house(2, x, v)) {
      const double vv = v[0] * v[0] + v[1] * v[1];
      const int k = hi - 1;
      for (int j = std::max(l, k - 1); j <= hi; ++j) {
        const double d = 2.0 * (v[0] * h(k, j) + v[1] * h(k + 1, j)) / vv;
        h(k, j) -= d * v[0];
        h(k + 1, j) -= d * v[1];
      }
      for (int i = l; i <= hi; ++i) {
        const double d = 2.0 * (h(i, k) * v[0] + h(i, k + 1) * v[1]) / vv;
        h(i, k) -= d * v[0];
        h(i, k + 1) -= d * v[1];
      }
    }
  }
  return 0;
}

// Arnoldi on Phi about the stored linearization: m steps, Ritz values sorted by modulus
// (largest first) into wr/wi [m]; the Hessenberg subdiagonal h_(m+1,m) into *hlast.
int floquet(pp_ctx* ctx, int m, double* wr, double* wi, double* hlast) {
  if (!ctx->lin_valid) return set_error(ctx, PP_ESTATE, "pp_floquet: no stored primal sweep");
  const int64_t n = ctx->ws_nu;
  if (m < 1 || m > n) return set_error(ctx, PP_EINVAL, "pp_floquet: m must lie in [1, N_u]");
  double* V = nullptr;
  double* d_h = nullptr;
  if (cudaMalloc(&V, sizeof(double) * (size_t)(m + 1) * n) != cudaSuccess ||
      cudaMalloc(&d_h, sizeof(double) * 72) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(V);
    return set_error(ctx, PP_ENOMEM, "pp_floquet: basis allocation failed");
  }
  struct Guard {
    double* a;
    double* b;
    ~Guard() {
      cudaFree(a);
      cudaFree(b);
    }
  } guard{V, d_h};
  std::vector<double> Hm((size_t)(m + 1) * m, 0.0), hc(m + 1), h(72);
  double* w = work_vec(ctx, 24);
  // deterministic start vector: all ones, normalized
  std::vector<double> ones(n, 1.0 / std::sqrt((double)n));
  PP_CK(cudaMemcpyAsync(V, ones.data(), sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
  PP_CK(cudaStreamSynchronize(ctx->stream));
  constexpr int CH = 64;  // columns per Gram-Schmidt chunk
  for (int j = 0; j < m; ++j) {
    const double* vj = V + (size_t)j * n;
    // w = Phi v_j = v_j - (I - Phi) v_j
    PP_TRY(tangent_sweep(ctx, vj, w));
    std::vector<double> coeffs{1.0, -1.0};
    const double* xs[2] = {vj, w};
    PP_CK(launch_lincomb<double>(n, w, 2, coeffs.data(), xs, ctx->stream));
    // two classical Gram-Schmidt passes against v_0..v_j, in chunks of CH columns
    std::fill(hc.begin(), hc.end(), 0.0);
    double nrm2 = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
      for (int c0 = 0; c0 <= j; c0 += CH) {
        const int kc = std::min(CH, j + 1 - c0);
        PP_CK(launch_mdot<double>(n, V + (size_t)c0 * n, n, kc, w, d_h, ctx->d_partial, ctx->d_counter,
                                  ctx->stream));
        PP_CK(launch_update_norm2<double>(n, V + (size_t)c0 * n, n, kc, d_h, w, d_h + CH, ctx->d_partial,
                                          ctx->d_counter, ctx->stream));
        PP_CK(cudaMemcpyAsync(h.data(), d_h, sizeof(double) * (CH + 1), cudaMemcpyDeviceToHost, ctx->stream));
        PP_CK(cudaStreamSynchronize(ctx->stream));
        for (int t = 0; t < kc; ++t) hc[c0 + t] += h[t];
        nrm2 = h[CH];
      }
    }
    const double hn = std::sqrt(std::max(nrm2, 0.0));
    for (int t = 0; t <= j; ++t) Hm[(size_t)t * m + j] = hc[t];
    if (!std::isfinite(hn)) return set_error(ctx, PP_ENAN, "pp_floquet: non-finite Arnoldi norm");
    if (j + 1 < m) Hm[(size_t)(j + 1) * m + j] = hn;
    if (j + 1 == m && hlast) *hlast = hn;
    if (hn == 0.0) {  // invariant subspace: the Ritz values of the leading block are exact
      m = j + 1;
      break;
    }
    PP_CK(launch_scale(n, V + (size_t)(j + 1) * n, 1.0 / hn, w, ctx->stream));
  }
  // Ritz values of the leading m x m block
  std::vector<double> Hs((size_t)m * m), r(m), im(m);
  for (int i = 0; i < m; ++i)
    for (int k = 0; k < m; ++k) Hs[(size_t)i * m + k] = Hm[(size_t)i * m + k];
  if (hessenberg_eigvals(m, Hs.data(), m, r.data(), im.data()) != 0)
    return set_error(ctx, PP_ENOCONV, "pp_floquet: Hessenberg QR did not converge");
  std::vector<int> ord(m);
  for (int i = 0; i < m; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(),
                   [&](int a, int b) { return std::hypot(r[a], im[a]) > std::hypot(r[b], im[b]); });
  for (int i = 0; i < m; ++i) {
    wr[i] = r[ord[i]];
    wi[i] = im[ord[i]];
  }
  return PP_OK;
}

}  // namespace pp

extern "C" {

int pp_hessenberg_eigvals(int n, double* H, int ld, double* wr, double* wi) {
  if (n < 1 || !H || !wr || !wi || ld < n) return PP_EINVAL;
  return pp::hessenberg_eigvals(n, H, ld, wr, wi) == 0 ? PP_OK : PP_ENOCONV;
}

int pp_floquet(pp_ctx* ctx, int m, double* wr, double* wi, double* hlast) {
  if (!ctx || !wr || !wi) return pp::set_error(ctx, PP_EINVAL, "pp_floquet: null argument");
  PP_CK(cudaSetDevice(ctx->device));
  return pp::floquet(ctx, m, wr, wi, hlast);
}

}  // extern "C"
