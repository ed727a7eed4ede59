// we_pipe3.cu -- the pipelined table SSA kernel compiled for 3 blocks per SM (few walker groups: the slowest group sets the launch (155 registers)).
#include "we_pipe.cuh"

namespace we {

cudaError_t launch_pipe_blocks3(const PropagateParams &prm, int groups, cudaStream_t st) {
  return launch_pipe_minb<3>(prm, groups, st);
}

}  // namespace we
