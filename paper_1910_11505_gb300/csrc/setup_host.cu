// Host-side setup math of the SG system: Karhunen-Loeve roots (Sec. 2.1, Eqs. gen_eigen and
// standard_deviation, in closed form for the separable exponential kernel), total-degree
// multi-index sets and Hermite triple products (Sec. 2.2), the 9-point Q1 pattern with its
// wavefront levels, and the operator work tables.
#include <algorithm>
#include <cmath>
#include <map>
#include <tuple>

#include "sg_internal.h"

namespace sg {

// ---------------------------------------------------------------- Karhunen-Loeve, 1-D

// On t in [-1/2, 1/2] with c = 1/ell the eigenfunctions of exp(-c|s-t|) are cos(w t) with
// c cos(w/2) = w sin(w/2), and sin(w t) with w cos(w/2) = -c sin(w/2).  Branch k of the even
// family has its root in (2k pi, (2k+1) pi), of the odd family in ((2k+1) pi, (2k+2) pi); both
// residual forms below are smooth and change sign exactly once in their bracket, so plain
// bisection down to adjacent doubles finds the root.
static double kl_residual(double w, double c, int odd) {
  return odd ? w * std::cos(0.5 * w) + c * std::sin(0.5 * w)
             : c * std::cos(0.5 * w) - w * std::sin(0.5 * w);
}

static double bisect(double lo, double hi, double c, int odd) {
  double flo = kl_residual(lo, c, odd);
  for (int it = 0; it < 4000; ++it) {
    double mid = 0.5 * (lo + hi);
    if (!(mid > lo && mid < hi)) break;
    double fm = kl_residual(mid, c, odd);
    if (fm == 0.0) return mid;
    if ((fm < 0) == (flo < 0)) {
      lo = mid;
      flo = fm;
    } else {
      hi = mid;
    }
  }
  return 0.5 * (lo + hi);
}

std::vector<KL1> kl_modes_1d(double ell, int count) {
  const double pi = 3.14159265358979323846;
  const double c = 1.0 / ell;
  std::vector<KL1> out;
  for (int k = 0; (int)out.size() < count; ++k) {
    for (int odd = 0; odd < 2 && (int)out.size() < count; ++odd) {
      double lo = (2 * k + odd) * pi, hi = (2 * k + odd + 1) * pi;
      double eps = 1e-14 * hi;
      double w = bisect(lo + eps, hi - eps, c, odd);
      KL1 m;
      m.w = w;
      m.odd = odd;
      m.mu = 2.0 * c / (w * w + c * c);
      m.nrm = std::sqrt(0.5 + (odd ? -1.0 : 1.0) * std::sin(w) / (2.0 * w));
      out.push_back(m);
    }
  }
  return out;
}

// 2-D terms of sigma^2 exp(-(|x1-y1| + |x2-y2|)/ell): products of 1-D pairs, largest M by
// eigenvalue, equal eigenvalues ordered by the (i, j) indices of their 1-D factors.
std::vector<KLTerm> kl_terms_2d(double sigma, double ell, int M) {
  std::vector<KL1> m1 = kl_modes_1d(ell, M + 1);
  std::vector<std::tuple<double, int, int>> cand;
  for (int i = 0; i < (int)m1.size(); ++i)
    for (int j = 0; j < (int)m1.size(); ++j) cand.emplace_back(-(m1[i].mu * m1[j].mu), i, j);
  std::sort(cand.begin(), cand.end());
  std::vector<KLTerm> out;
  for (int t = 0; t < M; ++t) {
    KLTerm term;
    term.i = std::get<1>(cand[t]);
    term.j = std::get<2>(cand[t]);
    term.fx = m1[term.i];
    term.fy = m1[term.j];
    term.lam = sigma * sigma * (-std::get<0>(cand[t]));
    term.sqrt_lam = std::sqrt(term.lam);
    out.push_back(term);
  }
  return out;
}

// ---------------------------------------------------------------- chaos index sets

static void rec_set(int M, int left, std::vector<int>& cur, std::vector<int>& out) {
  if ((int)cur.size() == M) {
    out.insert(out.end(), cur.begin(), cur.end());
    return;
  }
  for (int d = 0; d <= left; ++d) {
    cur.push_back(d);
    rec_set(M, left - d, cur, out);
    cur.pop_back();
  }
}

std::vector<int> total_degree_set(int M, int p) {
  std::vector<int> out, cur;
  rec_set(M, p, cur, out);
  return out;
}

// E[psi_i psi_j psi_k] of normalised Hermite polynomials under N(0,1): with s = (i+j+k)/2,
// sqrt(i! j! k!) / ((s-i)! (s-j)! (s-k)!) when s is an integer not below any of i, j, k.
double hermite_triple(int i, int j, int k) {
  int t = i + j + k;
  if (t & 1) return 0.0;
  int s = t / 2;
  if (s < i || s < j || s < k) return 0.0;
  auto fact = [](int v) {
    double r = 1.0;
    for (int x = 2; x <= v; ++x) r *= x;
    return r;
  };
  return std::sqrt(fact(i) * fact(j) * fact(k)) / (fact(s - i) * fact(s - j) * fact(s - k));
}

// ---------------------------------------------------------------- Q1 pattern and levels

Pattern make_pattern(int n) {
  Pattern pt;
  pt.n = n;
  pt.m = n + 1;
  const int m = pt.m;
  pt.N = m * m;
  pt.rowptr.assign(pt.N + 1, 0);
  for (int j = 0; j < m; ++j)
    for (int i = 0; i < m; ++i) {
      int r = i + m * j;
      for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) {
          int ii = i + di, jj = j + dj;
          if (ii < 0 || jj < 0 || ii >= m || jj >= m) continue;
          int c = ii + m * jj;
          if (c == r) pt.diag.push_back((int)pt.col.size());
          pt.col.push_back(c);
        }
      pt.rowptr[r + 1] = (int)pt.col.size();
    }
  pt.nnz = (int)pt.col.size();
  // forward levels: a row depends on the rows left of its diagonal
  std::vector<int> lf(pt.N, 0), lb(pt.N, 0);
  int nlf = 0, nlb = 0;
  for (int r = 0; r < pt.N; ++r) {
    int l = 0;
    for (int e = pt.rowptr[r]; e < pt.diag[r]; ++e) l = std::max(l, lf[pt.col[e]] + 1);
    lf[r] = l;
    nlf = std::max(nlf, l + 1);
  }
  for (int r = pt.N - 1; r >= 0; --r) {
    int l = 0;
    for (int e = pt.diag[r] + 1; e < pt.rowptr[r + 1]; ++e) l = std::max(l, lb[pt.col[e]] + 1);
    lb[r] = l;
    nlb = std::max(nlb, l + 1);
  }
  auto bucket = [&](const std::vector<int>& lev, int nl, std::vector<int>& ptr,
                    std::vector<int>& rows) {
    ptr.assign(nl + 1, 0);
    for (int r = 0; r < pt.N; ++r) ptr[lev[r] + 1]++;
    for (int l = 0; l < nl; ++l) ptr[l + 1] += ptr[l];
    rows.assign(pt.N, 0);
    std::vector<int> fill(ptr.begin(), ptr.end() - 1);
    for (int r = 0; r < pt.N; ++r) rows[fill[lev[r]]++] = r;
    for (int l = 0; l < nl; ++l) pt.max_width = std::max(pt.max_width, ptr[l + 1] - ptr[l]);
  };
  bucket(lf, nlf, pt.lev_f_ptr, pt.lev_f_rows);
  bucket(lb, nlb, pt.lev_b_ptr, pt.lev_b_rows);
  return pt;
}

int interior_level_width(int m) {
  int w = 0;
  for (int l = 3; l <= 3 * m - 6; ++l) {
    int y0 = std::max(1, (l - (m - 2) + 1) >> 1), y1 = std::min(m - 2, (l - 1) >> 1);
    w = std::max(w, y1 - y0 + 1);
  }
  return w;
}

}  // namespace sg
