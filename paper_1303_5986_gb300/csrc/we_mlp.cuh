// we_mlp.cuh -- host-side snapshot of a learned bin map (shared by we_mlp.cu and we_host.cu).
#pragma once
#include <cstdint>
#include <vector>

#include "../../include/we_ssa.h"

struct we_learned_bins {
  int n_in = 0, H = 0, n_bins = 0;
  std::vector<uint16_t> w1, w2, w3;     // BF16 bits
  std::vector<float> b1, b2, b3, zedges;
};

we_status make_learned_snapshot(const we_mlp *M, int32_t n_bins, const float *edges, we_learned_bins *L);
