// Cooperative multi-phase kernel and launcher for 1024x1024 images (field in global memory).
#define WF_LAUNCH_DEFINE_GLOBAL
#include "wf_launch.h"

namespace wf {
WF_INSTANTIATE_GLOBAL(1024)
}  // namespace wf
