// Host plan of one side's tiled split-CSR layout, computed from the row pointers alone: which
// rows are long, where every row's entries go, the chunks of the long rows, the staging stride,
// how many consecutive short tiles one walk item covers, and whether the FP64 walks sum a tile's
// longest rows warp-wide.  build_side uploads it; the C ABI
// exposes its summary (rhpdhg_plan_layout) so the rule can be checked without a GPU.
#pragma once

#include <cstdint>
#include <vector>

namespace rh {

struct SidePlan {
  int nrows = 0, ntiles = 0;
  std::vector<int> ptr_s;       // nrows: start of each row in the short arrays
  std::vector<int> tile_end;    // ntiles: end of each tile's short segment
  std::vector<int> dst;         // nrows: where each row's entries go (short or long arrays)
  std::vector<uint32_t> mask;   // ntiles: bit r set if row 32 t + r is long
  std::vector<int> long_rows, beg_l, end_l, chunk_ptr, chunk_row;
  long long nnz_s = 0, nnz_l = 0;   // padded lengths of the short and long arrays
  long long maxseg = 0;             // longest segment of one work item's tile group
  int mult = 1;                     // short tiles per work item
  int wide_rows = 0;                // FP64 walks sum a tile's longest rows warp-wide
  // longest segment of a work item's tile group with 1, 2 and 4 tiles per item (-1 where it
  // exceeds the staging budget): the walks the autotuner may choose instead of the rule's
  long long maxseg_mult[3] = {0, -1, -1};
};

// Plans the layout of a side with nrows rows and row pointers hp[0..nrows] (hp[0] = 0).
// Returns false when the padded arrays would not fit int32 offsets.
bool plan_side(const int *hp, int nrows, SidePlan *p);

}  // namespace rh
