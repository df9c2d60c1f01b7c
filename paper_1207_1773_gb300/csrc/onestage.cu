// onestage.cu -- one-stage comparator (paper Section 4.1).
#include "internal.cuh"

namespace gbhe {

size_t onestage_ws_bytes(int n, int m) { (void)n; (void)m; return 0; }

int hegv_onestage_run(Ctx& c, int n, cplx* A, int lda, cplx* B, int ldb, int il, int iu, double* w,
                      cplx* X, int ldx) {
  (void)c; (void)n; (void)A; (void)lda; (void)B; (void)ldb; (void)il; (void)iu; (void)w; (void)X; (void)ldx;
  return GBHE_ENOTCONV;
}

}  // namespace gbhe
