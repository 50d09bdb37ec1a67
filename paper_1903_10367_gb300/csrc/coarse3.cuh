// The bottom of the 3-D uniform path's coarse chain (coarse3.cu) with
// lmin = 1 in one launch: the restriction 2 -> 1 and the prolongations 1 -> 2
// and 2 -> 3, with the arithmetic of the separate launches (the same values).
#pragma once

#include "sweep3.cuh"

namespace adafac {

struct Bottom3Params {
  Level3Params r21;   // restriction to level 1 (r_f = r_2)
  Level3Params p12;   // prolongation to level 2 (g_f = g_2, t_f = t_2)
  Level3Params p23;   // prolongation to level 3 (g_f = g_3, t_f = t_3)
};
// levels 1, 2, 3 with 3, 9, 27 cells per axis
bool bottom3u_applies(const Bottom3Params& p);
void launch_bottom3u(const Bottom3Params& p, cudaStream_t s);

}  // namespace adafac
