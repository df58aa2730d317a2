// k_leaf_c16.cu -- leaf kernel instances with a 16-entry candidate list.
#include "k_leaf.cuh"

namespace bkd {
BKD_LEAF_DEFINE(16)
}  // namespace bkd
