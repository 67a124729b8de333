// Region plans: a GF(2^8) matrix M (rows x cols) cut into dense blocks for
// the region kernel, out[r] = sum_c M[r][c] * in[c] over byte blocks
// (Sec. 2: every operation of the code is Y = M X for some small M).
//
// Rows of a product-matrix generator that belong to the same slot j use the
// same inputs (the symbols of column j of the message matrix, Sec. 3.1), so
// grouping rows by their non-zero columns gives dense row x input blocks.
// Each input of a block is loaded and split once and then multiplied into
// every row of the block held in registers.
#pragma once
#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "code.h"

namespace pmrc {

constexpr int kMaxBlockRows = 16;   // rows held in registers per block
constexpr int kMaxSlots = 1024;     // input + output pointers per launch
// a matrix with more inputs + outputs than one launch takes, or a block of
// more than kPartCols x kMaxBlockRows coefficients (164 KiB of split tables
// in shared memory), is run as parts of at most kPartRows rows x kPartCols
// inputs
constexpr int kPartRows = 512;
constexpr int kPartCols = 512;

// Device image of one block (the arrays live in the same allocation).
struct BlockDesc {
  uint32_t in_off;    // index into the uint16 array: input slots
  uint32_t out_off;   // index into the uint16 array: output slots
  uint32_t tab_off;   // entry index into the split-table arrays (ninputs x R)
  uint16_t nrows;
  uint16_t ninputs;
};

// Split tables of one coefficient (see gf256.h): T0 and T1 as a 16-byte
// vector, T2 as one word.
struct TabEntry {
  uint32_t t0a, t0b, t1a, t1b;
};

struct PlanBlock {
  std::vector<uint16_t> rows;    // output slots
  std::vector<uint16_t> inputs;  // input slots
  std::vector<uint8_t> coef;     // inputs.size() x R, input-major
};

struct Plan;

// One launch of a plan too large for a single launch: rows `out_slots` of M
// restricted to the inputs `in_cols` (caller slot numbers).  The first part
// of a row set writes its outputs; the parts of later input chunks of the
// same rows XOR into them (accumulate), so they must run after it, in order.
struct PlanPart {
  std::shared_ptr<Plan> plan;
  std::vector<int> in_cols;
  std::vector<int> out_slots;
  bool accumulate = false;
};

struct Plan {
  int nin = 0, nout = 0;  // slots the caller supplies
  int R = 1;              // rows per block in the kernel (1, 2, 4, 8 or 16)
  int max_inputs = 0;     // largest block input count (shared-memory staging)
  int64_t nnz = 0;        // non-zero coefficients (work per byte)
  std::vector<PlanBlock> blocks;
  // BlockDesc[] | uint16 slots | TabEntry[] | uint32 T2[]
  std::vector<uint8_t> image;
  size_t idx_base = 0, tab4_base = 0, tab1_base = 0;
  int max_entries = 0;    // largest ninputs x R of a block
  // non-empty when nin + nout > kMaxSlots: the launches that replace `blocks`
  std::vector<PlanPart> parts;
  // per-device copies of `image`
  std::mutex mu;
  std::map<int, void *> dev;
  ~Plan();
  // Returns the device copy for the current device (uploads on first use).
  int device_image(const void **out, std::string &err);
};

// out_slot[r] is the output slot of row r (or -1 to skip the row).  Input
// slots are the columns of M; in the device image output slots are stored
// after them (slot index = M.cols + out_slot).  Above kMaxSlots slots the
// plan is cut into parts (see PlanPart).
std::shared_ptr<Plan> make_plan(const Mat &M, const std::vector<int> &out_slot, int nout);

// The input slots (columns of M) the plan reads, in increasing order.
std::vector<int> plan_reads(const Plan &p);

}  // namespace pmrc
