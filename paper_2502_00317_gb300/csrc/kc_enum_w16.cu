// kc_enum_w16.cu -- the enumerator kernels of width 16 (bitmap rows of 16 words),
// in a translation unit of their own so that the widths compile in parallel.
#include "kc_enum_dev.cuh"

namespace kc {
KC_DFS_DEF(16)
KC_TIER_KERNELS(16, 1)
}  // namespace kc
