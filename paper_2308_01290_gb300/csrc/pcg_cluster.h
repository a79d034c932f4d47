// Cluster-resident Z^m PCG (one slice per 16-CTA thread-block cluster).
#pragma once
#include <cstddef>

namespace recon {

struct Ctx;

constexpr int kClusterCtas = 16;
constexpr int kClusterThreads = 512;
constexpr size_t kClusterSmemMax = 225 * 1024;   // dynamic shared memory per CTA

// Picks the slices the cluster kernel can hold (FP32, width a multiple of 4,
// both sides >= 32, band and spectrum buffers within shared memory) and
// prepares the launch; no-op when none qualifies or clusters are unavailable.
int pcg_cluster_setup(Ctx& c);
// Runs the whole Z^m solve of every eligible active slice.
int pcg_cluster_run(Ctx& c);

}  // namespace recon
