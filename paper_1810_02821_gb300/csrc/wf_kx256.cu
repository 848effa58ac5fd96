// Cluster-resident hierarchical sampler (clusters of 4 CTAs of 64 rows) and spin-2 sampler (both
// components, clusters of 8 CTAs of 32 rows) for 256x256 images.
#define WF_LAUNCH_DEFINE_CLUSTER_EXT
#include "wf_launch.h"

namespace wf {
WF_INSTANTIATE_CLUSTER_BAND(256, 64)
WF_INSTANTIATE_CLUSTER_SPIN2(256, 32)
}  // namespace wf
