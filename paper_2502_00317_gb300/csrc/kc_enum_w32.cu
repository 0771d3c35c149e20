// kc_enum_w32.cu -- the enumerator kernels of width 32 (bitmap rows of 32 words),
// in a translation unit of their own so that the widths compile in parallel.
#include "kc_enum_dev.cuh"

namespace kc {
KC_DFS_DEF(32)
KC_TIER_KERNELS(32, 1)
}  // namespace kc
