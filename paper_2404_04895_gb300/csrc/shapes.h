// Construct-kernel launch shapes compiled into the library: (warps per ant,
// 16-byte chunks per lane).  A shape covers 32 * warps * chunks * V columns,
// V = 4 (fp32) or 8 (bf16 / fp16).  The row is staged in KC * 32 * W * 16
// bytes of shared memory, so an fp32 row may hold up to 49152 columns and a
// 16-bit row up to 65536.
#pragma once

#define ACO_SHAPES_4B(X) \
  X(1, 1) X(1, 2) X(1, 4) X(1, 8) X(1, 12) X(1, 16) X(1, 24) X(1, 32) X(1, 40) \
  X(2, 16) X(2, 20) X(2, 32) X(2, 40) X(4, 10) X(4, 16) X(4, 20) X(4, 32) X(8, 32) X(16, 24)

#define ACO_SHAPES_2B(X) \
  X(1, 1) X(1, 2) X(1, 4) X(1, 8) X(1, 12) X(1, 16) X(1, 20) X(1, 24) X(1, 32) \
  X(2, 8) X(2, 10) X(2, 16) X(2, 20) X(2, 32) X(4, 10) X(4, 16) X(4, 32) X(8, 32)
