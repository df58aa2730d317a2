// k_leaf_c12.cu -- leaf kernel instances with a 12-entry candidate list.
#include "k_leaf.cuh"

namespace bkd {
BKD_LEAF_DEFINE(12)
}  // namespace bkd
