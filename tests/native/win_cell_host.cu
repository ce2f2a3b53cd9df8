// Host program for tests/test_window_logic.py: reads cases "lo_x lo_y lo_z
// present c_x c_y c_z" (one per line) and prints the windowed query pass's
// decision for each: the window brick of the cell's lowest corner (-1 when
// the cell is not in the window), then, for an in-window cell, the window
// brick and in-brick slot of each of its 8 corners (corner k = dx + 2 dy + 4 dz).
#include <stdio.h>
#include <stdint.h>

#include "gp_query_win.cuh"

int main() {
  Win W;
  unsigned present;
  int c[3];
  while (scanf("%d %d %d %u %d %d %d", &W.lo[0], &W.lo[1], &W.lo[2], &present, &c[0], &c[1], &c[2]) == 7) {
    W.present = present;
    const int b0 = win_cell(W, c);
    printf("%d", b0);
    if (b0 >= 0) {
      for (int k = 0; k < 8; ++k) {
        int local;
        const int wb = win_corner(W, c, k & 1, (k >> 1) & 1, k >> 2, local);
        printf(" %d %d", wb, local);
      }
    }
    printf("\n");
  }
  return 0;
}
