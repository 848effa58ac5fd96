// Cluster-resident sampler and batch pipeline for 512x512 images (clusters of 16 CTAs of 32 rows).
#define WF_LAUNCH_DEFINE_CLUSTER
#include "wf_launch.h"

namespace wf {
WF_INSTANTIATE_CLUSTER(512, 32)
}  // namespace wf
