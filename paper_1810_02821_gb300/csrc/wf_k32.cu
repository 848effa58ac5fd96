// Kernels and launchers for 32x32 images.
#define WF_LAUNCH_DEFINE
#include "wf_launch.h"

namespace wf {
WF_INSTANTIATE(32)
}  // namespace wf
