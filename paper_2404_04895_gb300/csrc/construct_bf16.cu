// bf16 M_p instantiations of the tour-construction kernel.
#include "construct.cuh"
#include "internal.h"
#include "shapes.h"

namespace aco {

int launch_construct_bf16(const void* P, int n, int ld, int m, uint2 key, uint32_t it,
                          const uint32_t* it_dev, int32_t* tours, int32_t* err, int warps,
                          int chunks, int mode, const uint2* lists,
                         const int* lcnt, const uint32_t* lkey, cudaStream_t st) {
#define X(W, KC, MODE) ACO_CONSTRUCT_CASE(ACO_BF16, W, KC, MODE)
  ACO_SHAPES_2B(X)
#undef X
  return set_error(ACO_ERR_UNSUPPORTED, "construct shape (%d warps, %d chunks, mode %d) not compiled for bf16",
                   warps, chunks, mode);
}

int prepare_construct_bf16() {
#define X(W, KC, MODE) ACO_CONSTRUCT_PREPARE(ACO_BF16, W, KC, MODE)
  ACO_SHAPES_2B(X)
#undef X
  return ACO_OK;
}

int launch_batch_construct_bf16(const InstDev* insts, const int* ant_off, int count, int total,
                                int* counter, int32_t* err, int warps, int chunks, int mode,
                                int bitmap_bytes, int num_sms, cudaStream_t st) {
#define X(W, KC, MODE) ACO_BATCH_CONSTRUCT_CASE(ACO_BF16, W, KC, MODE)
  ACO_BATCH_SHAPES_2B(X)
#undef X
  return set_error(ACO_ERR_UNSUPPORTED, "batch construct shape (%d, %d, %d) not compiled", warps, chunks,
                   mode);
}

}  // namespace aco
