// Reduced-storage factor copies and their products (hodlr2d_mode other than
// F64).  Filled in by the float-float and mixed-precision paths.
#include "internal.h"

namespace h2d {

int prepare_mode(hodlr2d* h, int mode) {
  if (mode == HODLR2D_MODE_F64) return HODLR2D_OK;
  (void)h;
  return HODLR2D_ERR_STATE;
}

void free_modes(hodlr2d* h) {
  for (int l = 0; l < HODLR2D_MAX_LEVELS; ++l)
    for (int m = 0; m < 4; ++m) {
      cudaFree(h->lev[l].d_fac_mode[m]);
      h->lev[l].d_fac_mode[m] = nullptr;
    }
}

int matvec_mode_device(hodlr2d* h, const double* x, double* y, int nrhs, int mode) {
  (void)h; (void)x; (void)y; (void)nrhs; (void)mode;
  return HODLR2D_ERR_STATE;
}

}  // namespace h2d
