// Run-time specialised phase kernels (see jit.cpp).
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "kernels.hpp"
#include "planner.hpp"

namespace nwq {

// Run sweep sd of plan p through a kernel compiled for its structure.
// Returns false, launching nothing, when the sweep is not eligible (real
// plans, no phases, states below the size threshold, tables over the
// parameter or shared-memory budget) or NVRTC is unavailable or failed: the
// caller then runs the interpreted phase kernel.  When it returns true, *err
// holds the launch status.
// dw: the double-word kernel of the sweep (the state holds double words).
bool jit_launch_sweep(Plan& p, size_t sweep, const PhaseTables& pt, void* state, int sm_count, cudaStream_t s,
                      cudaError_t* err, bool dw = false);

// Double-word plans (p.dw): true when every sweep of p has a compiled
// double-word kernel (requesting the compiles as jit_launch_sweep does), so
// the plan can run with the state in the double-word layout.
bool jit_dw_ready(Plan& p);

// Source of the specialised kernel for sweep `sweep` of p (empty if not
// eligible) and its packed parameter bytes: a host-only hook for tests.
bool jit_source(const Plan& p, size_t sweep, std::string& src, size_t* param_bytes, size_t* smem_bytes);

// Host-only check: generate and compile (to cubin, nothing loaded) every
// eligible sweep of p; *eligible sweeps, *built compiled.  log: the first
// compiler error.
int jit_build_check(const Plan& p, int* eligible, int* built, std::string* log);

// Queue background compilation of every eligible sweep kernel of p that is
// not compiled yet; returns how many are pending.  Never waits.
int jit_prefetch(const Plan& p);

// Arithmetic of the plan's specialised kernels per state element, summed over
// the eligible sweeps (their count is returned): multiply-adds and multiplies
// of the kernels' value type, counted on the generated source (dw: the
// double-word kernels), and the arithmetic-pipe instructions they make.
int jit_plan_arith(const Plan& p, bool dw, double* fma_per_elem, double* mul_per_elem, double* instr_per_elem);

// States of at least this many index bits run specialised kernels (64: never).
int jit_min_state_bits();

// Stop the background compiler (queued kernels stay uncompiled; the one in
// progress finishes) and join its thread.  Idempotent.
void jit_shutdown();

// Kernels compiled so far in this process, and compile failures.
void jit_stats(int* compiled, int* failed);

}  // namespace nwq
