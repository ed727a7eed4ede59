// we_pipe4.cu -- the pipelined table SSA kernel compiled for 4 blocks per SM (many walker groups: the SMs' throughput sets the launch (128 registers)).
#include "we_pipe.cuh"

namespace we {

cudaError_t launch_pipe_blocks4(const PropagateParams &prm, int groups, cudaStream_t st) {
  return launch_pipe_minb<4>(prm, groups, st);
}

}  // namespace we
