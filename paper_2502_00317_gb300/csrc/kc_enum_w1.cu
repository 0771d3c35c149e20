// kc_enum_w1.cu -- the enumerator kernels of width 1 (bitmap rows of 1 word),
// in a translation unit of their own so that the widths compile in parallel.
#include "kc_enum_dev.cuh"

namespace kc {
KC_DFS_DEF(1)
KC_TIER_KERNELS(1, 1)
}  // namespace kc
