// Internal declarations shared by the host planner (plan.cpp) and the CUDA
// kernels (kernels.cu).  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/uw.h"

namespace uw {

// A captured product of an asynchronous host call, and everything its
// launches were built from: a call whose signature differs captures anew.
struct HostGraph {
  int fwd = 0, prec = 0, slot = 0, batch = 0, J0 = 0, line_variant = 0, coarse_mode = 0, grouped = 0;
  int64_t m = 0;
  const void *work = nullptr, *stage = nullptr, *mask = nullptr, *pos = nullptr;
  std::string env;        // the UW_* launch switches in force at capture
  bool tried = false;     // captured (or the capture was refused) for this signature
  void* exec = nullptr;   // cudaGraphExec_t; null after a refused capture: run eagerly
  bool same(const HostGraph& o) const {
    return fwd == o.fwd && prec == o.prec && slot == o.slot && batch == o.batch && J0 == o.J0 &&
           line_variant == o.line_variant && coarse_mode == o.coarse_mode && grouped == o.grouped && m == o.m &&
           work == o.work && stage == o.stage && mask == o.mask && pos == o.pos && env == o.env;
  }
};

// Device-side view of the input-independent tables, one copy per precision.
// Everything is indexed exactly like the host vectors of Plan below.
template <typename T>
struct Tables {
  const T* h;      // 2p            scaling filter h_k, k = -p+1..p
  const T* g;      // 2p            wavelet filter g_k = (-1)^k h_{1-k}
  const T* taps;   // (2p-1) Q      I_q[t] = int_{t/Q}^{(t+1)/Q} phi, t = (-p+1)Q ..
  const T* EL;     // p x (2p-1)Q   cell integrals of phi^left_m over [k/Q, (k+1)/Q)
  const T* ER;     // p x (2p-1)Q   cell integrals of phi^right_r over [-(k+1)/Q, -k/Q)
  const T* PL;     // p x Lb        level-1 coordinates of phi^left_m (Lb = 3p-1)
  const T* QL;     // p x Lb        level-1 coordinates of psi^left_m
  const T* PR;     // p x Lb        same on the right (coordinate c <-> index n1-1-c)
  const T* QR;     // p x Lb
};

// Per-kernel timing with CUDA events recorded on the launching stream around
// every launch (only while enabled): total time, launch count and the
// algorithmic bytes one launch must move (inputs read once, outputs written
// once).
struct Profiler;

// Geometry of the tensor-core (split-BF16) line operators of one plan (see
// tc_plan.cpp).  Forward: 16 consecutive outputs of H16 (T Syn) per block,
// from the lo / hi coefficients [bs n - W0, bs n - W0 + lw); adjoint: 8 lo and
// 8 hi outputs per block c from the partially transformed samples
// [16 Q c - W1, 16 Q c - W1 + 16 KSA).  Blocks next to a VMP boundary use
// small dense matrices instead (EBl / EBr forward, EAl / EAr adjoint blocks).
struct TcGeo {
  int ok = 0;
  int KS = 0, KSA = 0;      // k-steps (of 16) of the forward / adjoint block matrices
  int W0 = 0, lw = 0, bs = 0;
  int W1 = 0;
  int EBl = 0, EBr = 0, Xl = 0;   // forward edge blocks; inputs per side (lo and hi each, multiple of 4)
  int EAl = 0, EAr = 0, Wl = 0;   // adjoint edge blocks; inputs per side (multiple of 16)
  int SF = 0, SA = 0;       // row strides of the forward / adjoint edge matrices
  int HL = 0, HR = 0;       // forward halo (coefficients) left / right
  int HLa = 0, HRa = 0;     // adjoint halo (samples) left / right
  // word offsets into the device buffer d_tc
  int64_t oAf = 0, oAa = 0, oEf = 0, oEa = 0, words = 0;
};

// Edge corrections of the FP32 line operators (kernels_f32.cu).  The kernels
// apply the interior formulas of the last synthesis level and of T to the
// whole line with zero padding beyond its ends; near a VMP boundary the exact
// operator differs from that by a correction that reads only the p lo and p
// hi coefficients at that end and reaches only the first / last K outputs of
// T:  v_exact = v_interior + C x_edge.  C is K x 2p per side (rows v[0..K) on
// the left, v[N-K..N) on the right; columns lo[0..p), hi[0..p) on the left,
// lo[n0-p..n0), hi[n0-p..n0) on the right), rows padded to CS floats.  The
// adjoint adds C^T applied to the transformed samples at each end.
struct F32Geo {
  int ok = 0;
  int K = 0;       // corrected outputs of T per side (multiple of 16; 0 = periodic)
  int CS = 0;      // row stride of C (>= 2p, multiple of 4)
  int64_t words = 0;
};

// Geometry of the tcgen05 split-BF16 line operators (kernels_umma.cu), for
// lines of N = 4096 samples with q = 1.  A line is 128 blocks of 32 outputs,
// k = 32 b + r.  Forward: D1[b][r] = sum_j W[b][j] B1[r][j] with the window
// W[b][j] = lo[8 b - 8 + j] (j < 24), hi[8 b - 32 + j] (j >= 24), and B1 the
// last synthesis level, T and the Walsh-Hadamard stages of bits 0-4 of one
// block; the stages of bits 5-11 across the blocks follow on the CUDA
// cores.  The adjoint applies the transposes.  Near a VMP boundary the exact operator differs from the
// windowed interior one by a correction that reads only the p lo and p hi
// coefficients at that end and reaches only the first / last KB blocks.
// Device buffer d_umma: three BF16 parts of B1 (forward B operand, K-major,
// 32 x 48), three BF16 parts of B1^T (adjoint B operand, K-major, 48 x 32),
// then the corrections C'[2][KB * 32][2p] (FP32, the Walsh stages of bits
// 0-4 applied to each row block).
struct UmmaGeo {
  int ok = 0;
  int KB = 0;                  // corrected blocks per side (0: periodic or none)
  int64_t oF = 0, oA = 0;      // bf16 offsets of the operator parts (each 3 x 1536 values)
  int64_t oC = 0;              // float offset of the corrections
  int64_t bytes = 0;
};

struct Plan {
  int d = 1, R = 0, q = 0, p = 1, bd = 0, J0 = 0;
  int family = 0;            // 0: extremal-phase Daubechies, 1: least asymmetric (symlet)
  int M = 1, N = 1;          // per dimension
  int Q = 1, Lb = 2, ntap = 1;
  int64_t m = 0;             // samples
  int64_t words = 0;         // mask words (d = 1: ceil(N/32); d = 2: N * ceil(N/32))
  int wpr = 1;               // mask words per row
  int max_batch = 0;
  int last_launches = 0;

  // host tables (double, rounded from long double)
  std::vector<double> h, g, taps, EL, ER, PL, QL, PR, QR;

  // device memory
  void* d_tab64 = nullptr;   // packed double tables
  void* d_tab32 = nullptr;   // packed float tables
  Tables<double> t64{};
  Tables<float> t32{};
  uint32_t* d_mask = nullptr;    // words
  int32_t* d_prefix = nullptr;   // exclusive prefix count per word
  uint16_t* d_pos = nullptr;     // per sample (packed order): its natural FWHT position in the row (N <= 65536)
  int32_t* d_nat2y = nullptr;    // 1D, 2^13 <= N <= 2^22: natural FWHT position -> index of its sample in y, or -1
  void* d_work = nullptr;
  size_t work_bytes = 0;
  void* d_stage = nullptr;       // host-API staging: two slots of (input + output)
  size_t stage_bytes = 0;        // bytes per slot
  // asynchronous host calls: copy streams, per-slot events (upload done,
  // product done, download done), next slot
  void* s_up = nullptr;
  void* s_down = nullptr;
  void* ev[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
  int slot = 0;
  // the products of the asynchronous host calls as CUDA graphs, captured on
  // s_cap at first use and replayed while nothing they depend on changed
  void* s_cap = nullptr;
  std::vector<HostGraph> hgraphs;
  // launch choices (a plan group and its tuner set them): line operators
  // 0 = the fastest specialised kernel that applies, 1 = the generic kernels;
  // coarse 2D levels 0 = one cooperative launch, 1 = one launch per level
  int line_variant = 0;
  int coarse_mode = 0;
  void* group = nullptr;         // the live plan group that holds this plan (at most one)
  int device = 0;
  Profiler* prof = nullptr;
  TcGeo tc;                      // split-BF16 line operators (tc.ok = 0: not eligible)
  void* d_tc = nullptr;
  UmmaGeo umma;                  // tcgen05 line operators (umma.ok = 0: not eligible)
  void* d_umma = nullptr;
  F32Geo f32;                    // FP32 line operators (f32.ok = 0: not eligible)
  void* d_f32 = nullptr;         // [2][K][CS] floats (left, then right)
  void* d_sync = nullptr;        // grid barrier of the fused coarse-level kernels
  void* d_coarse = nullptr;      // coarse-level edge corrections: [2][Lb][2p] doubles, then floats
  int coarse_ok = 0;             // 1: the register-window coarse tiles may run
};

// plan.cpp
bool build_tables(Plan& P, std::string& err);
// tc_plan.cpp: block matrices of the tensor-core line operators (host, FP64);
// fills P.tc and the packed words to upload (empty if not eligible)
void build_tc(Plan& P, std::vector<uint32_t>& words);
// tc_plan.cpp: operator matrices and edge corrections of the tcgen05 line
// operators (host, FP64); fills P.umma and the bytes to upload (empty if not
// eligible)
void build_umma(Plan& P, std::vector<unsigned char>& bytes);
// tc_plan.cpp: edge corrections of the FP32 line operators (host, FP64);
// fills P.f32 and the floats to upload (empty if not eligible)
void build_f32(Plan& P, std::vector<float>& out);
// tc_plan.cpp: edge corrections of one 2D Mallat level, [2][Lb][2p] (empty
// for periodic plans); false if the boundary blocks do not have that structure
bool build_coarse(const Plan& P, std::vector<double>& D);
// group_kernel.cu: one persistent launch for the FP32 products of a plan
// group (NULL from pgroup_create, with the reason, if the group does not
// qualify); err: a device word set when a bounded wait gives up
struct PersistentGroup;
PersistentGroup* pgroup_create(const Plan* const* plans, int n, std::string& why);
int pgroup_run(PersistentGroup* g, bool fwd, const void* const* in, void* const* out, unsigned* err, void* stream);
int pgroup_set_params(PersistentGroup* g, int lines, int cols, int tiles, int rad, int ctas);
void pgroup_params(const PersistentGroup* g, int* p5);
void pgroup_destroy(PersistentGroup* g);
// kernels.cu
int upload_tables(Plan& P);
int launch_forward(const Plan& P, int prec, const void* x, void* y, int batch, void* stream, int* nlaunch);
int launch_adjoint(const Plan& P, int prec, const void* y, void* x, int batch, void* stream, int* nlaunch);
size_t workspace_bytes(const Plan& P, int batch);
void set_error(int status, const std::string& msg);
void profiler_free(Plan& P);

}  // namespace uw
