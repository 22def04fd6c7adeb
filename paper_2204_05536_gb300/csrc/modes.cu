// Factor copies per hodlr2d_mode and dispatch of the product by mode.
#include "internal.h"

namespace h2d {

int prepare_df32(hodlr2d* h);
int prepare_low(hodlr2d* h, int mode);
void free_v2(hodlr2d* h);
int product_device(hodlr2d* h, const double* x, double* y, int nrhs, int mode);

int prepare_mode(hodlr2d* h, int mode) {
  int rc = HODLR2D_OK;
  switch (mode) {
    case HODLR2D_MODE_F64: break;
    case HODLR2D_MODE_DF32: rc = prepare_df32(h); break;
    case HODLR2D_MODE_F32:
    case HODLR2D_MODE_BF16: rc = prepare_low(h, mode); break;
    default: return HODLR2D_ERR_ARG;
  }
  if (rc == HODLR2D_OK) h->prepared[mode] = true;
  return rc;
}

void free_modes(hodlr2d* h) {
  for (int l = 0; l < HODLR2D_MAX_LEVELS; ++l)
    for (int m = 0; m < 4; ++m) {
      cudaFree(h->lev[l].d_fac_mode[m]);
      h->lev[l].d_fac_mode[m] = nullptr;
    }
  free_v2(h);
}

int matvec_mode_device(hodlr2d* h, const double* x, double* y, int nrhs, int mode) {
  return product_device(h, x, y, nrhs, mode);
}

}  // namespace h2d
