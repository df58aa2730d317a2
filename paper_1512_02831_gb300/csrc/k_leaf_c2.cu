// k_leaf_c2.cu -- leaf kernel instances with a 2-entry candidate list.
#include "k_leaf.cuh"

namespace bkd {
BKD_LEAF_DEFINE(2)
}  // namespace bkd
