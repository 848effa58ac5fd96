// Cluster-resident hierarchical sampler and spin-2 sampler (both components) for 512x512 images,
// clusters of 16 CTAs of 32 rows.
#define WF_LAUNCH_DEFINE_CLUSTER_EXT
#include "wf_launch.h"

namespace wf {
WF_INSTANTIATE_CLUSTER_BAND(512, 32)
WF_INSTANTIATE_CLUSTER_SPIN2(512, 32)
}  // namespace wf
