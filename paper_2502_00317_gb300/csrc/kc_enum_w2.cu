// kc_enum_w2.cu -- the enumerator kernels of width 2 (bitmap rows of 2 words),
// in a translation unit of their own so that the widths compile in parallel.
#include "kc_enum_dev.cuh"

namespace kc {
KC_DFS_DEF(2)
KC_TIER_KERNELS(2, 1)
}  // namespace kc
