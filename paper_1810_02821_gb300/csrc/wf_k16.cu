// Kernels and launchers for 16x16 images.
#define WF_LAUNCH_DEFINE
#include "wf_launch.h"

namespace wf {
WF_INSTANTIATE(16)
}  // namespace wf
