// ck_insert_b4.cu -- the insert kernels of two-choice tables with 4-slot
// bins (every policy, with and without ghosts), in a translation unit of
// their own so that the library's kernels compile in parallel.
#include "ck_launch.cuh"

namespace ck {

InsertFn pick_insert_b4(uint32_t policy, bool ghost) { return pick_two_choice<4>(policy, ghost); }
InsertFn pick_insert_warp_b4() { return launch_insert_warp<4>; }

}  // namespace ck
