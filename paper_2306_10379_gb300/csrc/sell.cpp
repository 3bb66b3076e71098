// Host-side conversion of CSR to SELL-C-sigma (sliced ELLPACK with chunk
// height C and sorting window sigma). Integer layout work only; the values
// are copied, never combined.
#include <stdint.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "../../include/gsi.h"

extern "C" gsi_status gsi_sell_size(int64_t n, const int64_t* rowptr, int32_t C, int32_t sigma,
                                    int64_t* nchunks, int64_t* total) {
  if (n < 0 || !rowptr || C <= 0 || sigma <= 0 || !nchunks || !total) return GSI_ERR_ARG;
  int64_t nc = (n + C - 1) / C;
  // The chunk widths depend on the permutation; build it to size the arrays.
  std::vector<int64_t> perm(n);
  std::iota(perm.begin(), perm.end(), 0);
  for (int64_t w0 = 0; w0 < n; w0 += sigma) {
    int64_t w1 = std::min(n, w0 + sigma);
    std::stable_sort(perm.begin() + w0, perm.begin() + w1, [&](int64_t a, int64_t b) {
      return (rowptr[a + 1] - rowptr[a]) > (rowptr[b + 1] - rowptr[b]);
    });
  }
  int64_t tot = 0;
  for (int64_t ch = 0; ch < nc; ++ch) {
    int64_t width = 0;
    for (int64_t k = ch * C; k < std::min(n, (ch + 1) * C); ++k) {
      int64_t r = perm[k];
      width = std::max(width, rowptr[r + 1] - rowptr[r]);
    }
    tot += width * C;
  }
  *nchunks = nc;
  *total = tot;
  return GSI_OK;
}

extern "C" gsi_status gsi_csr_to_sell(int64_t n, const int64_t* rowptr, const int32_t* colidx,
                                      const double* val, int32_t C, int32_t sigma, int64_t* perm,
                                      int64_t* chunk_ptr, int64_t* chunk_len, int32_t* sell_col,
                                      double* sell_val) {
  if (n < 0 || !rowptr || C <= 0 || sigma <= 0 || !perm || !chunk_ptr || !chunk_len)
    return GSI_ERR_ARG;
  int64_t nc = (n + C - 1) / C;
  std::vector<int64_t> order(n);
  std::iota(order.begin(), order.end(), 0);
  // Inside each window: nnz descending; stable sort keeps ascending row index on ties.
  for (int64_t w0 = 0; w0 < n; w0 += sigma) {
    int64_t w1 = std::min(n, w0 + sigma);
    std::stable_sort(order.begin() + w0, order.begin() + w1, [&](int64_t a, int64_t b) {
      return (rowptr[a + 1] - rowptr[a]) > (rowptr[b + 1] - rowptr[b]);
    });
  }
  for (int64_t k = 0; k < nc * C; ++k) perm[k] = k < n ? order[k] : -1;
  chunk_ptr[0] = 0;
  for (int64_t ch = 0; ch < nc; ++ch) {
    int64_t width = 0;
    for (int64_t lane = 0; lane < C; ++lane) {
      int64_t r = perm[ch * C + lane];
      if (r >= 0) width = std::max(width, rowptr[r + 1] - rowptr[r]);
    }
    chunk_len[ch] = width;
    chunk_ptr[ch + 1] = chunk_ptr[ch] + width * C;
  }
  if (!sell_col || !sell_val) return GSI_OK;
  for (int64_t ch = 0; ch < nc; ++ch) {
    int64_t base = chunk_ptr[ch];
    for (int64_t lane = 0; lane < C; ++lane) {
      int64_t r = perm[ch * C + lane];
      int64_t len = r >= 0 ? rowptr[r + 1] - rowptr[r] : 0;
      for (int64_t j = 0; j < chunk_len[ch]; ++j) {
        int64_t slot = base + j * C + lane;
        if (j < len) {
          sell_col[slot] = colidx[rowptr[r] + j];
          sell_val[slot] = val[rowptr[r] + j];
        } else {
          sell_col[slot] = r >= 0 ? (int32_t)r : 0;
          sell_val[slot] = 0.0;
        }
      }
    }
  }
  return GSI_OK;
}
