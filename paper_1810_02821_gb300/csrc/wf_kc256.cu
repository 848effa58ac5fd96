// Cluster-resident sampler and batch pipeline for 256x256 images (clusters of 4 CTAs of 64 rows).
#define WF_LAUNCH_DEFINE_CLUSTER
#include "wf_launch.h"

namespace wf {
WF_INSTANTIATE_CLUSTER(256, 64)
}  // namespace wf
