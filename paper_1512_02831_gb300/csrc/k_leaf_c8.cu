// k_leaf_c8.cu -- leaf kernel instances with a 8-entry candidate list.
#include "k_leaf.cuh"

namespace bkd {
BKD_LEAF_DEFINE(8)
}  // namespace bkd
