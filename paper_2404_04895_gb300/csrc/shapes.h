// Construct-kernel launch shapes compiled into the library: (warps per ant,
// 16-byte chunks per lane, mode).  A shape covers 32 * warps * chunks * V
// columns, V = 4 (fp32) or 8 (bf16 / fp16).  Mode 1 (direct) keeps a step's
// chunks in registers: at most 12 per lane.  Mode 0 (staged) puts the row in
// KC * 32 * W * 16 bytes of shared memory, so an fp32 row may hold up to 49152
// columns and a 16-bit row up to 65536.
#pragma once

#define ACO_SHAPES_4B(X)                                                                        \
  X(1, 1, 1) X(1, 2, 1) X(1, 4, 1) X(1, 8, 1) X(1, 12, 1) X(2, 8, 1) X(2, 10, 1) X(2, 12, 1)   \
  X(4, 8, 1) X(4, 10, 1) X(4, 12, 1) X(8, 10, 1) X(8, 12, 1) X(16, 12, 1)                     \
  X(1, 16, 0) X(1, 24, 0) X(1, 32, 0) X(1, 40, 0) X(2, 20, 0) X(2, 32, 0) X(4, 20, 0)          \
  X(4, 32, 0) X(8, 32, 0) X(16, 24, 0)

#define ACO_SHAPES_2B(X)                                                                        \
  X(1, 1, 1) X(1, 2, 1) X(1, 4, 1) X(1, 8, 1) X(1, 10, 1) X(1, 12, 1) X(2, 8, 1) X(2, 10, 1)  \
  X(2, 12, 1) X(4, 10, 1) X(4, 12, 1) X(8, 12, 1)                                              \
  X(1, 16, 0) X(1, 20, 0) X(1, 32, 0) X(2, 16, 0) X(2, 20, 0) X(4, 16, 0) X(8, 32, 0)

// Shapes of the multi-instance (persistent) construction kernel; a batch
// groups its instances into size classes, one shape (and launch) per class.
#define ACO_BATCH_SHAPES_4B(X)                                                                 \
  X(1, 1, 1) X(1, 2, 1) X(1, 4, 1) X(1, 8, 1) X(1, 12, 1) X(2, 8, 1) X(2, 12, 1) X(4, 10, 1)   \
  X(4, 12, 1) X(4, 20, 0) X(8, 32, 0)

#define ACO_BATCH_SHAPES_2B(X)                                                                 \
  X(1, 1, 1) X(1, 2, 1) X(1, 4, 1) X(1, 8, 1) X(1, 12, 1) X(2, 8, 1) X(2, 10, 1) X(4, 10, 1)   \
  X(4, 12, 1) X(4, 16, 0) X(8, 32, 0)
