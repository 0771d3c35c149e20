// kc_enum_w4.cu -- the enumerator kernels of width 4 (bitmap rows of 4 words),
// in a translation unit of their own so that the widths compile in parallel.
#include "kc_enum_dev.cuh"

namespace kc {
KC_DFS_DEF(4)
KC_TIER_KERNELS(4, 1)
}  // namespace kc
