// k_leaf_c4.cu -- leaf kernel instances with a 4-entry candidate list.
#include "k_leaf.cuh"

namespace bkd {
BKD_LEAF_DEFINE(4)
}  // namespace bkd
