// Kernels and launchers for 64x64 images.
#define WF_LAUNCH_DEFINE
#include "wf_launch.h"

namespace wf {
WF_INSTANTIATE(64)
}  // namespace wf
