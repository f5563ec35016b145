// ck_insert_b1.cu -- the insert kernels of d-ary tables with single-slot
// bins (random kicking, rattle-kicking and the searches), in a translation
// unit of their own so that the library's kernels compile in parallel.
#include "ck_launch.cuh"

namespace ck {

InsertFn pick_insert_b1(uint32_t policy) {
  switch (policy) {
    case CK_RATTLE: return launch_insert<1, P_RATTLE, false>;
    case CK_BFS: return launch_insert<1, P_BFS, false>;
    case CK_SORTED: return launch_insert<1, P_SORTED, false>;
    case CK_HYBRID: return launch_insert<1, P_HYBRID, false>;
    default: return launch_insert<1, P_RANDOM, false>;
  }
}

}  // namespace ck
