// Candidate lists of M_p (the exact fast path of the construction step): the
// sizes and the marker the list builders (steps.cuh) write and the
// construction kernels read.  A row's list holds its ACO_LIST_TARGET largest
// entries (ties at the cut in column order, at most ACO_LIST_MAX), sorted by
// value; slots past the count hold (0, kListPad).
#pragma once

#include <stdint.h>

#include "tensoraco.h"

namespace aco {

constexpr int kListTarget = ACO_LIST_TARGET;
constexpr int kListMax = ACO_LIST_MAX;
constexpr uint32_t kListPad = 0xFFFFFFFFu;  // column of the slots past the count

}  // namespace aco
