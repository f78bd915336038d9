// Handles behind the opaque ABI types (internal to the library).
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <memory>

#include "planner.hpp"

struct nwq_plan {
  nwq::Plan p;
};

struct nwq_state {
  int kind = 0, n = 0, dtype = 0, B = 0;
  void* buf = nullptr;
  size_t bytes = 0;
  bool owned = false;
  // The buffer holds the double-word layout a double-word plan run left there
  // (library-owned FP64 states only; every FP64 reader converts it back first).
  bool dw_resident = false;
  bool dw_exact = false;  // resident pairs normalised (a reset or a renormalisation wrote them)
  cudaStream_t stream = nullptr;
  int device = 0, sm_count = 1;
  std::unique_ptr<nwq_plan> p2r, r2p;                // DM conversions
  std::map<double, std::unique_ptr<nwq_plan>> probs;  // readout / transform plans keyed by e
};

namespace nwq {
// Record msg as the calling thread's last error and return code.
int set_error(int code, const char* msg);
}  // namespace nwq
