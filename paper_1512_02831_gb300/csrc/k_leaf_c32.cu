// k_leaf_c32.cu -- leaf kernel instances with a 32-entry candidate list.
#include "k_leaf.cuh"

namespace bkd {
BKD_LEAF_DEFINE(32)
}  // namespace bkd
