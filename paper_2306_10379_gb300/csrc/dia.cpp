// Host-side diagonal layout of a CSR matrix whose nonzeros lie on a few
// diagonals (the finite-difference stencils): the distinct offsets
// col - row, ascending, and the values by row and diagonal (zero where the
// matrix has no entry). Integer layout work and copies; entries repeated in
// a row are summed.
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "../../include/gsi.h"

extern "C" gsi_status gsi_csr_to_dia(int64_t n, const int64_t* rowptr, const int32_t* colidx,
                                     const double* val, int32_t max_diags, int32_t* ndiag,
                                     int64_t* offsets, double* dia) {
  if (n < 0 || !rowptr || !ndiag || max_diags < 1 || (n > 0 && !colidx)) return GSI_ERR_ARG;
  if (rowptr[0] != 0) return GSI_ERR_ARG;
  std::vector<int64_t> offs;
  for (int64_t r = 0; r < n; ++r) {
    if (rowptr[r + 1] < rowptr[r]) return GSI_ERR_ARG;
    for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) {
      if (colidx[k] < 0 || colidx[k] >= n) return GSI_ERR_ARG;
      const int64_t o = (int64_t)colidx[k] - r;
      if (std::find(offs.begin(), offs.end(), o) == offs.end()) {
        offs.push_back(o);
        if ((int64_t)offs.size() > max_diags) {
          *ndiag = 0;  // not stencil-shaped within max_diags
          return GSI_OK;
        }
      }
    }
  }
  std::sort(offs.begin(), offs.end());
  *ndiag = (int32_t)offs.size();
  if (offsets)
    for (size_t d = 0; d < offs.size(); ++d) offsets[d] = offs[d];
  if (dia && val) {
    const int64_t nd = (int64_t)offs.size();
    std::fill(dia, dia + n * nd, 0.0);
    for (int64_t r = 0; r < n; ++r)
      for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) {
        const int64_t d = std::lower_bound(offs.begin(), offs.end(), (int64_t)colidx[k] - r) - offs.begin();
        dia[r * nd + d] += val[k];
      }
  }
  return GSI_OK;
}
