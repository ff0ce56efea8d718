// NVRTC options of the tiled pass kernels, shared by the in-process compile
// (tile_jit.cpp) and the compile worker (worker/nvrtc_worker.cpp), so both
// produce the same cubin for the same source.
#pragma once

namespace sv {

inline const char *const kPassNvrtcOpts[] = {"--gpu-architecture=sm_103a", "--std=c++17", "--ptxas-options=-v"};
constexpr int kPassNvrtcOptsQuiet = 2;    // the first two
constexpr int kPassNvrtcOptsVerbose = 3;  // with ptxas resource usage in the log

}  // namespace sv
