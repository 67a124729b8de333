// Internal view of the code handle, shared by the C ABI and the batching
// and serving layers.
#pragma once
#include <condition_variable>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "bitslice.h"
#include "code.h"
#include "plan.h"
#include "repair.h"
#include "specific.h"

namespace pmrc {

// One compilation of a run-time schedule (host only), shared by the handle
// and the thread that runs it.
struct BsJob {
  std::mutex mu;
  std::condition_variable cv;
  bool done = false;
  int rc = 0;
  std::string err;
  BsCompiled out;
};

}  // namespace pmrc

struct pmrc_code {
  pmrc::CodeMatrices m;
  std::shared_ptr<pmrc::Plan> encode;  // built at create
  int bs_id = -1;                      // generated bitsliced encode kernel, or -1
  int encode_kernel = 0;               // PMRC_KERNEL_*
  mutable std::mutex mu;               // guards cache
  mutable std::map<std::string, std::shared_ptr<pmrc::Plan>> cache;
  mutable std::map<std::string, std::shared_ptr<pmrc::FusedRepairPlan>> fused;
  mutable std::map<std::string, std::shared_ptr<pmrc::SpecificPlan>> specific;
  // bitsliced kernels compiled at run time: reconstruction rows per (nodes,
  // wanted rows), newcomer applies per (failed node, helpers), the encode
  // ("e"); a null kernel records a matrix that could not be built
  int decode_kernel = 0;                    // PMRC_KERNEL_*
  mutable std::map<std::string, std::shared_ptr<pmrc::BsRuntimeKernel>> rt;
  mutable std::map<std::string, std::string> rt_err;
  // compilations in flight (background under PMRC_KERNEL_AUTO), per key;
  // the first call that finds one finished loads it into `rt`
  mutable std::map<std::string, std::shared_ptr<pmrc::BsJob>> rt_jobs;
  // evicted run-time kernels stay loaded until the handle is destroyed: a
  // launch from them may still be running
  mutable std::vector<std::shared_ptr<pmrc::BsRuntimeKernel>> rt_retired;
  // reconstructions of a systematic code: per (nodes, wanted rows), the
  // estimated ALU work per 32-byte column of the one-launch schedule and of
  // the two-launch factored one (-1: not possible), decided at first use
  mutable std::map<std::string, std::pair<long long, long long>> decode_costs;
};

namespace pmrc {

constexpr size_t kPlanCacheCap = 4096;

void set_last_error(const std::string &msg);

std::shared_ptr<Plan> cached_plan(const pmrc_code *c, const std::string &key,
                                  const std::function<std::shared_ptr<Plan>()> &make);
int helper_plan(const pmrc_code *c, int f, int nh, std::shared_ptr<Plan> &out, std::string &err);
int newcomer_plan(const pmrc_code *c, int f, const int *helpers, std::shared_ptr<Plan> &out,
                  std::string &err);
int decode_plan(const pmrc_code *c, const int *nodes, const std::vector<char> &want,
                std::shared_ptr<Plan> &out, std::string &err);
int fused_repair_plan(const pmrc_code *c, int f, const int *helpers,
                      std::shared_ptr<FusedRepairPlan> &out, std::string &err);
int decode_wanted(const pmrc_code *c, const int *nodes, const uint8_t *const *node_blocks,
                  uint8_t *const *data_out, std::vector<char> &want);

}  // namespace pmrc
