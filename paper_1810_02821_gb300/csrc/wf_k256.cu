// Cooperative multi-phase kernel and launcher for 256x256 images (field in global memory).
#define WF_LAUNCH_DEFINE_GLOBAL
#include "wf_launch.h"

namespace wf {
WF_INSTANTIATE_GLOBAL(256)
}  // namespace wf
