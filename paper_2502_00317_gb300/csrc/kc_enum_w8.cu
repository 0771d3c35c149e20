// kc_enum_w8.cu -- the enumerator kernels of width 8 (bitmap rows of 8 words),
// in a translation unit of their own so that the widths compile in parallel.
#include "kc_enum_dev.cuh"

namespace kc {
KC_DFS_DEF(8)
KC_TIER_KERNELS(8, 1)
}  // namespace kc
