// Matrix features for the learned blocking (host, production).  The paper
// observes that the better blocking and its parameter depend on the matrix
// (block-size sweeps, Table 2; resolution dependence, Sec. 6.1); these
// statistics of the sparsity pattern and values are the inputs of the model
// that predicts them.  Definitions (row degree = stored entries of the row,
// diagonal included; off-diagonal count = degree minus the diagonal):
//   0  log10(n)                  1  mean row degree
//   2  variance of row degree    3  skewness of row degree (0 when the variance is 0)
//   4  largest row degree        5  log10(nnz)
//   6  mean of min(d_i, 10), d_i = |a_ii| / sum_{j != i} |a_ij| (rows without
//      off-diagonal entries: d_i = 10)
//   7  min_i min(d_i, 10)        8  fraction of rows with d_i >= 1
//   9  max |i - j| / n over stored entries (bandwidth)
//  10  mean |i - j| / n over off-diagonal entries (0 if none)
//  11-18  fractions of rows whose off-diagonal count lies in [0,2], [3,4], [5,6],
//      [7,8], [9,12], [13,20], [21,40], [41, inf)
//  19  min(log10(max |a_ij| / min |a_ij|) over nonzero off-diagonal values, 6)
//      (0 if there are none)
// Sums run over rows in ascending order, entries in stored order.
#include <algorithm>
#include <cmath>

#include "iccg_internal.h"

extern "C" iccg_status iccg_features(int32_t n, const int64_t *rowptr, const int32_t *colind, const double *val,
                                     double out[ICCG_NFEATURES]) {
  if (n < 1 || !rowptr || !colind || !val || !out) return ICCG_ERR_ARG;
  const int64_t nnz = rowptr[n];
  if (rowptr[0] != 0 || nnz < 0) return ICCG_ERR_ARG;
  for (int32_t i = 0; i < n; ++i)
    if (rowptr[i + 1] < rowptr[i]) return ICCG_ERR_ARG;
  for (int64_t e = 0; e < nnz; ++e)
    if (colind[e] < 0 || colind[e] >= n) return ICCG_ERR_ARG;
  for (int k = 0; k < ICCG_NFEATURES; ++k) out[k] = 0.0;
  const double dn = double(n);
  double s1 = 0.0, dmax = 0.0;
  for (int32_t i = 0; i < n; ++i) {
    const double d = double(rowptr[i + 1] - rowptr[i]);
    s1 += d;
    dmax = std::max(dmax, d);
  }
  const double mean = s1 / dn;
  double m2 = 0.0, m3 = 0.0;
  for (int32_t i = 0; i < n; ++i) {
    const double d = double(rowptr[i + 1] - rowptr[i]) - mean;
    m2 += d * d;
    m3 += d * d * d;
  }
  m2 /= dn;
  m3 /= dn;
  out[0] = std::log10(dn);
  out[1] = mean;
  out[2] = m2;
  out[3] = m2 > 0.0 ? m3 / std::pow(m2, 1.5) : 0.0;
  out[4] = dmax;
  out[5] = std::log10(std::max(double(nnz), 1.0));
  double dsum = 0.0, dmin = 10.0, ndom = 0.0, band = 0.0, prof = 0.0, noff_tot = 0.0;
  double vmax = 0.0, vmin = INFINITY;
  static const int edges[8] = {2, 4, 6, 8, 12, 20, 40, 1 << 30};
  double hist[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int32_t i = 0; i < n; ++i) {
    double diag = 0.0, off = 0.0;
    int64_t noff = 0;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const int32_t j = colind[e];
      const double a = std::fabs(val[e]);
      const double dist = double(j > i ? j - i : i - j);
      band = std::max(band, dist);
      if (j == i) {
        diag += a;
      } else {
        off += a;
        ++noff;
        prof += dist;
        if (a > 0.0) {
          vmax = std::max(vmax, a);
          vmin = std::min(vmin, a);
        }
      }
    }
    const double di = off > 0.0 ? std::min(diag / off, 10.0) : 10.0;
    dsum += di;
    dmin = std::min(dmin, di);
    ndom += di >= 1.0 ? 1.0 : 0.0;
    noff_tot += double(noff);
    int b = 0;
    while (noff > edges[b]) ++b;
    hist[b] += 1.0;
  }
  out[6] = dsum / dn;
  out[7] = dmin;
  out[8] = ndom / dn;
  out[9] = band / dn;
  out[10] = noff_tot > 0.0 ? prof / noff_tot / dn : 0.0;
  for (int b = 0; b < 8; ++b) out[11 + b] = hist[b] / dn;
  out[19] = vmax > 0.0 ? std::min(std::log10(vmax / vmin), 6.0) : 0.0;
  return ICCG_OK;
}
