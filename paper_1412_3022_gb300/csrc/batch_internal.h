// Work lists of the persistent kernel in batch.cu, shared by the batched
// API (pmrc_batch_*) and the serving loop (serve.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "plan.h"
#include "repair.h"

struct pmrc_code;

namespace pmrc {

// One stripe operation, ready to be cut into work items.
struct WorkStripe {
  int type = 0;  // 0: region plan (encode, decode), 1: fused repair
  std::shared_ptr<Plan> plan;
  std::shared_ptr<FusedRepairPlan> fplan;
  std::vector<uint8_t *> ptrs;  // inputs, then outputs (device pointers)
  size_t nbytes = 0;
  int64_t user_bytes = 0;       // k*alpha*B (encode, decode) or alpha*B (repair)
  int64_t work = 0;             // products per byte column (cost model)
  bool aligned = true;
};

int stripe_encode(const pmrc_code *c, const uint8_t *const *data, uint8_t *const *out,
                  size_t nbytes, WorkStripe &s, std::string &err);

// An encode large enough to run as its own launch of the code's built-in
// bitsliced kernel (beside the batched kernel, in the same graph or
// iteration): bytes [0, nbytes) of every block, nbytes a multiple of 32;
// a ragged tail of the stripe stays with the batched kernel.
struct BitslicedEncode {
  int id = -1;  // built-in kernel (bitslice_find)
  std::vector<const uint8_t *> in;
  std::vector<uint8_t *> out;
  size_t nbytes = 0;
};

// Stripes of at least this many data bytes (k alpha x B) take the bitsliced
// launch: below it the batched kernel's fine-grained items beat a launch.
constexpr size_t kBatchBitslicedMinBytes = 4u << 20;

// Whether an encode of c over nbytes-byte blocks takes its bitsliced kernel
// (built-in kernel, GF(2^8), at least kBatchBitslicedMinBytes of data,
// every pointer non-NULL and 16-byte aligned); fills e when it does.
bool bitsliced_encode_split(const pmrc_code *c, const uint8_t *const *data, uint8_t *const *out,
                            size_t nbytes, BitslicedEncode &e);
int stripe_repair(const pmrc_code *c, int f, const int *helpers, const uint8_t *const *blocks,
                  uint8_t *const *out, size_t nbytes, WorkStripe &s, std::string &err);
int stripe_decode(const pmrc_code *c, const int *nodes, const uint8_t *const *node_blocks,
                  uint8_t *const *data_out, size_t nbytes, WorkStripe &s, std::string &err);

// Device work item (position independent: pointers are offsets into the
// launch's pointer table).  The kernel reads it as four 16-byte words, so
// the list may sit in device memory or in mapped pinned host memory.
struct alignas(16) WorkItem {
  const uint8_t *image;    // region plan image or fused repair image (device)
  uint64_t nbytes;         // block size of the stripe
  uint32_t ptr_off;        // first pointer of the stripe in the table
  uint32_t nptrs;          // pointers of the stripe (inputs, then outputs)
  uint32_t tile0, ntiles;  // tile range: 4 KiB tiles (region), 1 KiB (fused repair)
  uint32_t idx_base, tab4_base, tab1_base;  // region image offsets
  uint16_t type;           // 0 region block, 1 fused repair
  uint16_t block;          // region: block index
  uint16_t stride;         // region: table stride (the plan's R)
  uint16_t aligned;
  uint32_t reserved;
};
static_assert(sizeof(WorkItem) == 64, "work items are read as four 16-byte words");

struct WorkList {
  std::vector<uint8_t *> ptrs;
  std::vector<WorkItem> items;
  size_t smem = 64;        // dynamic shared memory per CTA (pointer area included)
  size_t ptr_area = 0;     // leading bytes of it holding the item's stripe pointers
  int64_t user_bytes = 0;
};

// Items per persistent CTA the work list is cut for: an item costs at most
// 1/(kItemsPerCta x CTAs) of the list, so the last items pulled leave the
// grid's tail short.
constexpr int kItemsPerCta = 4;

// Appends the stripes' items (biggest stripes first, blocks of one tile
// range adjacent) and pointers; plan images are uploaded on first use.
// Items span work_bytes of each block, or fewer tiles where one item would
// cost more than 1/target_items of all the stripes' products (target_items
// <= 0: no limit).
int worklist_build(const std::vector<const WorkStripe *> &stripes, int work_bytes,
                   int target_items, WorkList &wl, std::string &err);

// Persistent CTAs per SM that fit the kernel with this shared memory.
int worklist_ctas_per_sm(size_t smem);

// Counter reset + persistent kernel over nitems items.  items and ptrs are
// device-accessible: device memory, or mapped pinned host memory that the
// kernel reads in place (one item and its stripe's pointers per pull);
// ptr_area is the WorkList's.
cudaError_t worklist_launch(const WorkItem *items, int nitems, uint8_t *const *ptrs,
                            unsigned *d_counter, unsigned grid, size_t smem, size_t ptr_area,
                            cudaStream_t stream);

}  // namespace pmrc
