// Kernels and launchers for 128x128 images.
#define WF_LAUNCH_DEFINE
#include "wf_launch.h"

namespace wf {
WF_INSTANTIATE(128)
}  // namespace wf
