// Choice of the collide-and-stream kernel for one update (launch_step): the
// wall kernel for bounded grids; for 16-bit stores the direct paired kernel
// for the even update and the staged row-segment kernel for the odd one where
// the row length allows, else the whole-row kernel; otherwise (and for FP32
// stores) one thread per cell. Kept apart from the kernels so that a change of
// routing leaves their sources, and the profiles keyed to them, unchanged.
#include "lbrr_launch.h"

namespace lbrr {

cudaError_t launch_step(int q, int storage, int model, void *f, const Grid &g, float om1,
                        int parity, int *status, cudaStream_t st) {
  if (g.walls) return launch_step_walls(q, storage, model, f, g, om1, parity, st);
  if (storage != 0) {
    if (parity == 0 && pair16_even_supported(g))
      return launch_step_pair16_even(q, storage, model, f, g, om1, st);
    if (parity == 1 && tiled16_supported(g))
      return launch_step_tiled16_odd(q, storage, model, f, g, om1, st);
    bool launched = false;
    cudaError_t e = launch_step_row16(q, storage, model, f, g, om1, parity, status, st, launched);
    if (e != cudaSuccess || launched) return e;
  }
  return launch_step_cell(q, storage, model, f, g, om1, parity, st);
}

}  // namespace lbrr
