// Fused single-node repair (repair.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "code.h"

namespace pmrc {

// Device image: header, then split tables (stage 1: nz entries for phi_f's
// non-zeros; stage 2, lane-major: entry (q, lane l, m) at nz + q*4*rl + l*rl
// + m holds D[l + 4m][q], rl = ceil(alpha / 4); see repair_dev.cuh).
struct FusedRepairHeader {
  uint32_t d, alpha, nz, direct;
  uint32_t tab4_off, tab1_off;
  uint32_t rl, pad;
  uint16_t nzidx[16];  // which of a helper's alpha blocks phi_f reads
};

struct FusedRepairPlan {
  FusedRepairHeader header;
  std::vector<uint8_t> image;
  std::mutex mu;
  std::map<int, void *> dev;
  ~FusedRepairPlan();
  int device_image(const void **out, std::string &err);
};

std::shared_ptr<FusedRepairPlan> make_fused_repair_plan(const std::vector<uint8_t> &phi,
                                                        const Mat &D);

// CTAs of a fused repair launch over ntiles 1 KiB tiles.
unsigned fused_repair_grid(uint32_t ntiles);

// Shared memory of one CTA: the d x 1 KiB projections and the split tables.
size_t fused_repair_smem(const FusedRepairHeader &h);

// Runs the repair.  helper_blocks: d*alpha pointers, out: alpha pointers.
// The plan's tables are uploaded to the device on first use.
int launch_fused_repair(FusedRepairPlan &plan, const uint8_t *const *helper_blocks,
                        uint8_t *const *out, size_t nbytes, cudaStream_t stream,
                        std::string &err);

// Same repair with the tables copied into a fixed array compiled into the
// library instead of an uploaded plan; allocates no device memory (see
// pmrc_repair_noalloc in include/pmrc.h).
int launch_fused_repair_noalloc(const FusedRepairPlan &plan, const uint8_t *const *helper_blocks,
                                uint8_t *const *out, size_t nbytes, cudaStream_t stream,
                                std::string &err);

}  // namespace pmrc
