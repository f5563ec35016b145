// ck_insert_b8.cu -- the insert kernels of two-choice tables with 8-slot
// bins (every policy, with and without ghosts), in a translation unit of
// their own so that the library's kernels compile in parallel.
#include "ck_launch.cuh"

namespace ck {

InsertFn pick_insert_b8(uint32_t policy, bool ghost) { return pick_two_choice<8>(policy, ghost); }
InsertFn pick_insert_warp_b8() { return launch_insert_warp<8>; }

}  // namespace ck
