// Prints, for the single-precision compile-time plans whose forward column kernel copies
// its layer tiles with tensor copies, the byte offsets of every model column's tile in the
// kernel's shared memory for every layer row count ny (fwd_tile_stride), and for the
// bulk-copy row kernels the byte offsets of the rows_c2r input rows (c2r_in_row) for every
// transform length of the menu.  A CPU test checks their alignment.  Host code only.
#include <stdio.h>

#include "../../paper_2004_13904_gb300/csrc/tf_ct_kernels.cuh"

int main() {
  using tfk::ctk::fwd_tile_stride;
  using tfk::ctk::c2r_in_row;
  constexpr int TB = 8, MC = 2;   // the forward column kernel's tiles (ColTiles, FwdTmem)
  for (int ny = 1; ny <= 256; ++ny)
    for (int c = 0; c < MC; ++c)
      printf("tile %d %d %zu %d\n", ny, c, (size_t)c * fwd_tile_stride<float2, TB>(ny) * sizeof(float2),
             ny * TB * (int)sizeof(float2));
  constexpr int RT = 2 * tfk::ctk::PipeTiles::TB;
  for (int n1 = 258; n1 <= 512; n1 += 2) {
    const int hs = (n1 / 2 + 1 + 15) / 16 * 16;
    for (int r = 0; r <= RT; ++r)
      printf("c2r %d %d %d %zu\n", n1, hs, r, (size_t)c2r_in_row<RT>(r, hs) * sizeof(float2));
  }
  return 0;
}
