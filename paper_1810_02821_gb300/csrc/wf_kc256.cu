// Cluster-resident sampler for 256x256 images (field in the distributed shared memory of one cluster).
#define WF_LAUNCH_DEFINE_CLUSTER
#include "wf_launch.h"

namespace wf {
WF_INSTANTIATE_CLUSTER(256)
}  // namespace wf
