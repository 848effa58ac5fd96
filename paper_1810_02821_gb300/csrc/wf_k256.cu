// Cooperative multi-phase kernel and launcher for 256x256 images (field in global memory).
#define WF_LAUNCH_DEFINE_GLOBAL
// scalar FP32 here: with the paired forms the shared-memory FFT kernels spill (measured 20-30% slower)
#define WF_NO_F32X2 1
#include "wf_launch.h"

namespace wf {
WF_INSTANTIATE_GLOBAL(256)
}  // namespace wf
