// Cooperative multi-phase kernel and launcher for 512x512 images (field in global memory).
#define WF_LAUNCH_DEFINE_GLOBAL
#include "wf_launch.h"

namespace wf {
WF_INSTANTIATE_GLOBAL(512)
}  // namespace wf
