// k_leaf_c64.cu -- leaf kernel instances with a 64-entry candidate list.
#include "k_leaf.cuh"

namespace bkd {
BKD_LEAF_DEFINE(64)
}  // namespace bkd
