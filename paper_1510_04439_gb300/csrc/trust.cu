// Derivative-free trust-region bandwidth search (Section 3.3).
//
// Section 3.3 minimises the noisy cross-validation score over the bandwidth
// vector with the trust-region method of Marazzi and Nocedal, the local model
// fitted by quadratic regression instead of interpolation.  Host-side driver
// around the batched CV smoother (fpca_smooth_cov_project): every iteration
// sends its new sample bandwidths to the GPU in one launch sequence.
//
// Steps (variables x = log h, d <= 2, box [log h_lo, log h_hi]^d):
//  * trust region |x - x_k|_inf <= Delta_k; sample the 3^d stencil
//    x_k + Delta_k v, v in {-1, 0, 1}^d (lexicographic, clipped to the box,
//    duplicates dropped), CV values cached by point;
//  * least-squares fit of q(u) = c + g'u + u'Hu/2, u = (x - x_k)/Delta_k, to the
//    finite values (normal equations, Cholesky); too few finite values: Delta/2;
//  * step: exact minimiser of q over the trust-region box intersected with the
//    bounds, by enumerating the active sets (each coordinate free, at its lower
//    or at its upper bound; a free block's stationary point kept when feasible;
//    smallest value, first on ties);
//  * pred = q(0) - q(u) <= 0: Delta/2; else rho = (f(x_k) - f(x_t)) / pred,
//    accept when rho >= 0.1; rho < 0.25: Delta/2; rho > 0.75 with |u|_inf > 0.99:
//    Delta = min(2 Delta, Delta_max);
//  * stop when Delta < Delta_min or after max_iter iterations; the result is the
//    best point evaluated (lowest finite CV, first on ties).
#include <cmath>
#include <cstring>
#include <vector>

#include "fpca_internal.cuh"

namespace {

constexpr int TR_DMAX = 2;
constexpr int TR_NPAR = (TR_DMAX + 1) * (TR_DMAX + 2) / 2;

struct Pt {
  double x[TR_DMAX];
};

bool same(const Pt& a, const Pt& b, int d) {
  for (int k = 0; k < d; ++k)
    if (a.x[k] != b.x[k]) return false;
  return true;
}

// regression row: 1, u_k, then u_i u_j / 2 (i == j) or u_i u_j (i < j)
int quad_row(const double* u, int d, double* row) {
  int k = 0;
  row[k++] = 1.0;
  for (int i = 0; i < d; ++i) row[k++] = u[i];
  for (int i = 0; i < d; ++i)
    for (int j = i; j < d; ++j) row[k++] = i == j ? 0.5 * u[i] * u[i] : u[i] * u[j];
  return k;
}

// Solve the SPD system A x = b (n <= TR_NPAR) by Cholesky; false if not SPD.
bool chol_solve(int n, double A[TR_NPAR][TR_NPAR], double* b) {
  double L[TR_NPAR][TR_NPAR] = {};
  for (int j = 0; j < n; ++j) {
    double s = A[j][j];
    for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
    if (!(s > 0.0)) return false;
    L[j][j] = std::sqrt(s);
    for (int i = j + 1; i < n; ++i) {
      double v = A[i][j];
      for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
      L[i][j] = v / L[j][j];
    }
  }
  for (int i = 0; i < n; ++i) {
    double v = b[i];
    for (int k = 0; k < i; ++k) v -= L[i][k] * b[k];
    b[i] = v / L[i][i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double v = b[i];
    for (int k = i + 1; k < n; ++k) v -= L[k][i] * b[k];
    b[i] = v / L[i][i];
  }
  return true;
}

struct Quad {
  double c, g[TR_DMAX], H[TR_DMAX][TR_DMAX];
  double value(const double* u, int d) const {
    double v = c;
    for (int i = 0; i < d; ++i) {
      v += g[i] * u[i];
      for (int j = 0; j < d; ++j) v += 0.5 * u[i] * H[i][j] * u[j];
    }
    return v;
  }
};

// argmin over lo <= u <= hi of g'u + u'Hu/2, d <= 2, by enumerating active sets
bool box_qp(const Quad& q, const double* lo, const double* hi, int d, double* best_u) {
  double best = INFINITY;
  bool found = false;
  const int nstate = d == 1 ? 3 : 9;
  for (int st = 0; st < nstate; ++st) {
    int state[TR_DMAX];  // 0 free, 1 lower, 2 upper; first coordinate varies slowest
    for (int k = d - 1, r = st; k >= 0; --k, r /= 3) state[k] = r % 3;
    double u[TR_DMAX] = {0.0, 0.0};
    int free_[TR_DMAX], nf = 0, bound[TR_DMAX], nb = 0;
    for (int k = 0; k < d; ++k) {
      if (state[k] == 0) {
        free_[nf++] = k;
      } else {
        u[k] = state[k] == 1 ? lo[k] : hi[k];
        bound[nb++] = k;
      }
    }
    if (nf > 0) {
      double rhs[TR_DMAX];
      double hmax = 0.0;
      for (int a = 0; a < nf; ++a) {
        rhs[a] = -q.g[free_[a]];
        for (int b = 0; b < nb; ++b) rhs[a] -= q.H[free_[a]][bound[b]] * u[bound[b]];
        for (int b = 0; b < nf; ++b) hmax = std::fmax(hmax, std::fabs(q.H[free_[a]][free_[b]]));
      }
      const double scale = std::pow(std::fmax(1.0, hmax), (double)nf);
      if (nf == 1) {
        const double h = q.H[free_[0]][free_[0]];
        if (std::fabs(h) < 1e-12 * scale) continue;
        u[free_[0]] = rhs[0] / h;
      } else {
        const double a = q.H[0][0], b = q.H[0][1], c = q.H[1][0], e = q.H[1][1];
        const double det = a * e - b * c;
        if (std::fabs(det) < 1e-12 * scale) continue;
        u[0] = (rhs[0] * e - b * rhs[1]) / det;
        u[1] = (a * rhs[1] - c * rhs[0]) / det;
      }
      bool feasible = true;
      for (int a = 0; a < nf; ++a) {
        const int k = free_[a];
        if (u[k] < lo[k] - 1e-12 || u[k] > hi[k] + 1e-12) feasible = false;
      }
      if (!feasible) continue;
    }
    double v = 0.0;
    for (int i = 0; i < d; ++i) {
      v += q.g[i] * u[i];
      for (int j = 0; j < d; ++j) v += 0.5 * u[i] * q.H[i][j] * u[j];
    }
    if (v < best) {
      best = v;
      found = true;
      for (int k = 0; k < d; ++k) best_u[k] = u[k];
    }
  }
  return found;
}

struct Search {
  fpca_ctx* ctx;
  const fpca_grid* grid;
  const fpca_covbins* bins;
  int prec, d;
  double* dcv;  // device scratch, 9 doubles
  std::vector<Pt> pts;
  std::vector<double> vals;

  // values at the points (new ones evaluated in one batch, in order)
  fpca_status evaluate(const std::vector<Pt>& want, std::vector<double>& out) {
    std::vector<Pt> fresh;
    for (const Pt& p : want) {
      bool known = false;
      for (const Pt& q : pts) known = known || same(p, q, d);
      for (const Pt& q : fresh) known = known || same(p, q, d);
      if (!known) fresh.push_back(p);
    }
    if (!fresh.empty()) {
      std::vector<double> h(fresh.size() * d);
      for (size_t i = 0; i < fresh.size(); ++i)
        for (int k = 0; k < d; ++k) h[i * d + k] = std::exp(fresh[i].x[k]);
      fpca_status s = fpca_smooth_cov_project(ctx, grid, bins, h.data(), (int)fresh.size(), prec,
                                              nullptr, nullptr, 0, nullptr, nullptr, nullptr, dcv);
      if (s != FPCA_OK) return s;
      std::vector<double> cv(fresh.size());
      if (cudaMemcpyAsync(cv.data(), dcv, sizeof(double) * fresh.size(), cudaMemcpyDeviceToHost,
                          ctx->stream) != cudaSuccess)
        return fpca_fail(ctx, FPCA_E_CUDA, "reading the CV scores");
      s = fpca_sync(ctx);
      if (s != FPCA_OK) return s;
      for (size_t i = 0; i < fresh.size(); ++i) {
        pts.push_back(fresh[i]);
        vals.push_back(cv[i]);
      }
    }
    out.clear();
    for (const Pt& p : want)
      for (size_t i = 0; i < pts.size(); ++i)
        if (same(p, pts[i], d)) {
          out.push_back(vals[i]);
          break;
        }
    return FPCA_OK;
  }
};

}  // namespace

extern "C" fpca_status fpca_bw_trust_region(fpca_ctx* ctx, const fpca_grid* grid,
                                            const fpca_covbins* bins, int prec, const double* h0,
                                            const fpca_tr_options* opt, double* h_best,
                                            double* cv_best, int* n_evals, double* trace,
                                            int trace_cap) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  // host-driven: every iteration reads its CV values back
  if (fpca_no_capture(ctx, "fpca_bw_trust_region") != FPCA_OK) return FPCA_E_UNSUPPORTED;
  if (!grid || grid->d < 1 || grid->d > TR_DMAX)
    return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "the trust-region search is built for d <= 2");
  if (!bins || !h0 || !h_best)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "bins, h0 and h_best are required");
  fpca_tr_options o{0.4, 0.01, 1.0, 0.02, 0.6, 20};
  if (opt) o = *opt;
  if (!(o.h_lo > 0.0 && o.h_hi > o.h_lo && o.delta0 > 0.0 && o.delta_min > 0.0 &&
        o.delta_max >= o.delta0 && o.max_iter >= 0))
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "inconsistent trust-region options");
  const int d = grid->d;
  Search S{ctx, grid, bins, prec, d, nullptr, {}, {}};
  if (cudaMalloc(&S.dcv, sizeof(double) * 9) != cudaSuccess)
    return fpca_fail(ctx, FPCA_E_OOM, "CV scratch");
  double lo[TR_DMAX], hi[TR_DMAX];
  Pt x{};
  for (int k = 0; k < d; ++k) {
    lo[k] = std::log(o.h_lo);
    hi[k] = std::log(o.h_hi);
    x.x[k] = std::fmin(std::fmax(std::log(h0[k]), lo[k]), hi[k]);
  }
  fpca_status st = FPCA_OK;
  std::vector<double> v;
  double delta = o.delta0, fx = 0.0;
  st = S.evaluate({x}, v);
  if (st == FPCA_OK) {
    fx = v[0];
    if (!std::isfinite(fx))
      st = fpca_fail(ctx, FPCA_E_INVALID_ARG, "the starting bandwidth has an infinite CV score");
  }
  const int npar = (d + 1) * (d + 2) / 2;
  for (int it = 0; st == FPCA_OK && it < o.max_iter; ++it) {
    if (delta < o.delta_min) break;
    std::vector<Pt> sp;
    const int nst = d == 1 ? 3 : 9;
    for (int s = 0; s < nst; ++s) {
      Pt p{};
      for (int k = d - 1, r = s; k >= 0; --k, r /= 3) {
        const double vk = (double)(r % 3) - 1.0;  // -1, 0, 1
        p.x[k] = std::fmin(std::fmax(x.x[k] + delta * vk, lo[k]), hi[k]);
      }
      bool dup = false;
      for (const Pt& q : sp) dup = dup || same(p, q, d);
      if (!dup) sp.push_back(p);
    }
    st = S.evaluate(sp, v);
    if (st != FPCA_OK) break;
    double AtA[TR_NPAR][TR_NPAR] = {}, Aty[TR_NPAR] = {};
    int nfin = 0;
    for (size_t i = 0; i < sp.size(); ++i) {
      if (!std::isfinite(v[i])) continue;
      double u[TR_DMAX], row[TR_NPAR];
      for (int k = 0; k < d; ++k) u[k] = (sp[i].x[k] - x.x[k]) / delta;
      quad_row(u, d, row);
      for (int a = 0; a < npar; ++a) {
        Aty[a] += row[a] * v[i];
        for (int b = 0; b < npar; ++b) AtA[a][b] += row[a] * row[b];
      }
      ++nfin;
    }
    if (nfin < npar || !chol_solve(npar, AtA, Aty)) {
      delta *= 0.5;
      continue;
    }
    Quad q{};
    q.c = Aty[0];
    for (int k = 0; k < d; ++k) q.g[k] = Aty[1 + k];
    for (int i = 0, k = 1 + d; i < d; ++i)
      for (int j = i; j < d; ++j, ++k) q.H[i][j] = q.H[j][i] = Aty[k];
    double ulo[TR_DMAX], uhi[TR_DMAX], u[TR_DMAX] = {0.0, 0.0}, zero[TR_DMAX] = {0.0, 0.0};
    for (int k = 0; k < d; ++k) {
      ulo[k] = std::fmax(-1.0, (lo[k] - x.x[k]) / delta);
      uhi[k] = std::fmin(1.0, (hi[k] - x.x[k]) / delta);
    }
    const bool found = box_qp(q, ulo, uhi, d, u);
    const double pred = found ? q.value(zero, d) - q.value(u, d) : -INFINITY;
    if (!(pred > 0.0)) {
      delta *= 0.5;
      continue;
    }
    Pt xt{};
    double umax = 0.0;
    for (int k = 0; k < d; ++k) {
      xt.x[k] = x.x[k] + delta * u[k];
      umax = std::fmax(umax, std::fabs(u[k]));
    }
    st = S.evaluate({xt}, v);
    if (st != FPCA_OK) break;
    const double ft = v[0];
    const double rho = std::isfinite(ft) ? (fx - ft) / pred : -INFINITY;
    if (rho >= 0.1) {
      x = xt;
      fx = ft;
    }
    if (rho < 0.25)
      delta *= 0.5;
    else if (rho > 0.75 && umax > 0.99)
      delta = std::fmin(2.0 * delta, o.delta_max);
  }
  cudaFree(S.dcv);
  if (st != FPCA_OK) return st;
  int ib = -1;
  for (size_t i = 0; i < S.vals.size(); ++i)
    if (std::isfinite(S.vals[i]) && (ib < 0 || S.vals[i] < S.vals[ib])) ib = (int)i;
  for (int k = 0; k < d; ++k) h_best[k] = std::exp(S.pts[ib].x[k]);
  if (cv_best) *cv_best = S.vals[ib];
  if (n_evals) *n_evals = (int)S.vals.size();
  if (trace)
    for (int i = 0; i < (int)S.vals.size() && i < trace_cap; ++i) {
      for (int k = 0; k < d; ++k) trace[i * (d + 1) + k] = std::exp(S.pts[i].x[k]);
      trace[i * (d + 1) + d] = S.vals[i];
    }
  return FPCA_OK;
}
