// ozaki.cu -- split-precision (Ozaki-style) trailing update for DD.
#include <cuda_runtime.h>
#include "mw_common.cuh"
#include "lu_internal.cuh"

namespace mw {

size_t split_workspace_bytes(int64_t n, int nb) {
  (void)n;
  (void)nb;
  return 0;
}

int split_update_dd(double* A, int64_t lda, int64_t plane, int64_t row0, int64_t m, int64_t col0,
                    int64_t N, int64_t k0, int nb, char* ws, size_t ws_bytes, cudaStream_t s) {
  (void)A; (void)lda; (void)plane; (void)row0; (void)m; (void)col0; (void)N; (void)k0; (void)nb;
  (void)ws; (void)ws_bytes; (void)s;
  return MW_EUNSUPPORTED;
}

}  // namespace mw
