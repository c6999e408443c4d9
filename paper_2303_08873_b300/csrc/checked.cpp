// Status of the bounds-check build: reads the device words that AR_CHK
// (common.cuh) keeps per source file.
#include <cstdint>

#include "ar.h"
#include "ar_loops.h"

namespace ar {
int chk_read_daxpy(unsigned int* out2, int clear);
int chk_read_jacobi7(unsigned int* out2, int clear);
int chk_read_spmv(unsigned int* out2, int clear);
int chk_read_nbody(unsigned int* out2, int clear);
int chk_read_executor(unsigned int* out2, int clear);
int chk_read_mlp(unsigned int* out2, int clear);
int chk_read_peaks(unsigned int* out2, int clear);
}  // namespace ar

extern "C" int ar_check_status(int* enabled, uint32_t* first_failure, uint32_t* failures, int clear) {
  if (!enabled || !first_failure || !failures) return AR_ERR_ARG;
#ifdef AR_CHECKED
  *enabled = 1;
#else
  *enabled = 0;
#endif
  int (*const readers[])(unsigned int*, int) = {ar::chk_read_daxpy, ar::chk_read_jacobi7, ar::chk_read_spmv,
                                                ar::chk_read_nbody, ar::chk_read_executor, ar::chk_read_mlp,
                                                ar::chk_read_peaks};
  uint32_t first = 0, count = 0;
  for (auto rd : readers) {
    unsigned int w[2] = {0u, 0u};
    if (rd(w, clear) != 0) return AR_ERR_CUDA;
    if (!first && w[0]) first = w[0];
    count += w[1];
  }
  *first_failure = first;
  *failures = count;
  return AR_OK;
}
