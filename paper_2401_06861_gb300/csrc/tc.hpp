// Dense five-qubit blocks on the tensor cores (complex64 state vectors):
// types shared by the host planner (tc_plan.cpp) and the kernel (tc_kernels.cu).
//
// A block is a 32 x 32 complex matrix U on qubits q[0] < ... < q[4] (local
// index bit i <-> qubit q[i]).  As a real contraction over interleaved
// (re, im) pairs it is a 64 x 64 real matrix M, and one pass over the state
// computes, for every setting of the other qubits, y = M x over the 64 reals
// of that column: a GEMM D[m][n] = sum_k A[m][k] B[n][k] with A = the state
// columns (128 per tile) and B = M, run as tcgen05 MMAs of kind TF32 with
// the three-term split hi*hi + hi*lo + lo*hi (FP32-level accuracy).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <complex>
#include <vector>

namespace nwq {

constexpr int kTcBits = 5;       // qubits per block
constexpr int kTcRowBits = 7;    // other qubits per tile: 128 rows of the MMA
constexpr int kTcTileBits = 12;  // 2^12 amplitudes (32 KiB) per tile
constexpr int kTcMinQubits = kTcTileBits;
constexpr int kTcMaxFree = 34 - kTcTileBits;
constexpr size_t kTcMatFloats = 2 * 64 * 64;  // TF32 hi and lo parts of M, row-major

// Tile geometry of one block, computed on the host and passed by value.
struct TcGeom {
  uint64_t gw[kTcTileBits];  // amplitude offset of tile bit p (tile qubits ascending)
  uint64_t fw[kTcMaxFree];   // amplitude offset of bit b of the tile index
  uint32_t sw[kTcTileBits];  // shared-memory byte offset of tile bit p in the operand layout (XOR-combined)
  uint32_t ntiles;           // 2^(n - 12)
  // 1 when thread t's lane and warp bits are the row bits m0..m6 in order and its loop
  // steps the K chunks j1..j4 (blocks with no qubit below 4): its accumulator lane t then
  // holds exactly the amplitudes it loaded, which it stores back without a shared-memory pass
  uint32_t direct;
};

struct TcBlock {
  int q[kTcBits] = {0, 0, 0, 0, 0};
  std::vector<std::complex<double>> U;  // 32 x 32, row-major
  int gate0 = 0, ngates = 0;
};

// Geometry of a block on qubits q (ascending) of an n-qubit state.
void tc_geometry(const int* q, int n, TcGeom& g);
// hi / lo TF32 parts of the real 64 x 64 form of U (out: kTcMatFloats floats).
void tc_matrix_tables(const TcBlock& b, float* out);
// One pass of one block over the state (psi: 2^n complex64, in place).
// wait_test: withhold the MMAs so every MMA-completion wait runs out (test of
// the bounded waits; the tiles are left unwritten).
cudaError_t launch_tc_block(void* psi, const TcGeom& g, const float* mats_dev, int sm_count, cudaStream_t s,
                            bool wait_test = false);
// Number of bounded waits that ran out in the tensor-core kernel since the
// library was loaded on the current device (0 in a healthy run; synchronises).
cudaError_t tc_timeouts(int* count);

}  // namespace nwq
