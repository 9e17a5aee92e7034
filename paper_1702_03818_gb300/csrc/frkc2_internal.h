// Internal declarations shared by the FRKC2 host code and kernels (not part of the C ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "frkc2.h"

struct frkc2_plan_s {
  int s = 0;
  double beta = 0.0;
  double Q = 0.0;
  int n_iter = 0;
  std::vector<int> order;     // root index of each stage
  std::vector<double> a_re;   // step sizes in stage order
  std::vector<double> a_im;
  bool paired = false;        // conjugates adjacent: stages 2p, 2p+1 form one real pair
  double gain = 0.0;          // rounding gain of the stage order (frkc2_plan_rounding_gain)
};

namespace frkc2 {

// NVTX range for the enclosing scope (host timeline: a call, a step, a pass; no cost without a
// tool attached)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr int KMAX = 16;                 // most stages in one pass
constexpr unsigned ST_NONFINITE = 1u;    // status word bits
constexpr unsigned ST_TIMEOUT = 2u;
constexpr unsigned ST_BOUNDS = 4u;       // bounds-checking build: an index left its array

// Index checks of the bounds-checking build (FRKC2_DEBUG_BOUNDS, libfrkc2_debug.so): false
// and ST_BOUNDS latched in *status when ok is false, the caller then skipping the access.  In
// the normal build it is the constant true and the check compiles away.
#ifdef FRKC2_DEBUG_BOUNDS
__device__ __forceinline__ bool in_bounds(bool ok, unsigned* status) {
  if (!ok) atomicOr(status, ST_BOUNDS);
  return ok;
}
#else
__device__ __forceinline__ constexpr bool in_bounds(bool, unsigned*) { return true; }
#endif

// state layouts a pass reads or writes (the streaming pass honours them; the tile kernels
// always use planar U, V)
constexpr int PASS_IO_REAL = 0;     // U only (imaginary part zero on input, dropped on output)
constexpr int PASS_IO_PLANAR = 1;   // separate U and V arrays
constexpr int PASS_IO_COMPLEX = 2;  // one interleaved (U, V) array at U_in / U_out

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// One k-stage pass over the grid: read (U, V), apply k stages, write (U, V).
struct PassArgs {
  int ndim, bc;
  int nx, ny, nz;         // grid extents (1 past ndim)
  int tx, ty, tz;         // output tile of one CTA
  int hx, hy, hz;         // halo width per axis: k along present axes, 0 otherwise
  int k;                  // stages in this pass
  int check_finite;       // flag non-finite outputs in the status word
  int in_mode, out_mode;  // PASS_IO_* (streaming pass only)
  const void* U_in;       // real part of the pass input
  const void* V_in;       // imaginary part; nullptr = zero (first pass of a step)
  void* U_out;
  void* V_out;            // nullptr = not stored (last pass of a step)
  const void* H_in;       // embedded first-order solution (tile kernel only); nullptr = none
  void* H_out;
  const void* fx;         // face conductivities (FIELD / CONST), layouts in faces_layout()
  const void* fy;
  const void* fz;
  double kc, kp;          // POWER: kappa(w) = 1 + kc * w^kp
  unsigned* status;
  double ca[KMAX];        // dt Re(a_l) / dx^2 for the pass's stages
  double cb[KMAX];        // dt Im(a_l) / dx^2
  float caf[KMAX];        // the same, rounded to float once on the host
  float cbf[KMAX];
};

// Face arrays: x faces [nz][ny][nx+1], y faces [nz][ny+1][nx], z faces [nz+1][ny][nx];
// face index i along an axis lies between cells i-1 and i.
struct FaceLayout {
  size_t nfx, nfy, nfz;   // element counts (0 for absent axes)
};
FaceLayout faces_layout(const frkc2_problem& p);

// Workspace layout of frkc2_step (byte offsets from the workspace base).
struct StepLayout {
  size_t status, fx, fy, fz, fen, ua, va, ub, vb, total;
};
StepLayout step_layout(const frkc2_problem& p);

size_t state_bytes(int precision);
size_t arith_bytes(int precision);
size_t cells(const frkc2_problem& p);

// Launchers (return cudaGetLastError()).
cudaError_t launch_faces(const frkc2_problem& p, void* fx, void* fy, void* fz, cudaStream_t st);
cudaError_t launch_rho(const frkc2_problem& p, const void* u, double* rho_dev, cudaStream_t st);
cudaError_t launch_pass_generic(const frkc2_problem& p, const PassArgs& a, cudaStream_t st);
cudaError_t launch_err_sum(const frkc2_problem& p, const void* u, const void* h, double* out, cudaStream_t st);
cudaError_t launch_pass_stream2d(const frkc2_problem& p, const PassArgs& a, const void* fen, cudaStream_t st);
size_t face_pair_bytes(const frkc2_problem& p);
cudaError_t launch_face_pairs(const frkc2_problem& p, const void* fx, const void* fy, void* out, cudaStream_t st);
// overlap_previous: the launch may start while the previous launch on the stream (a pass of
// the same kind) finishes; its CTAs read the pass input only after that launch completes.
cudaError_t launch_pass_tb2d(const frkc2_problem& p, const PassArgs& a, cudaStream_t st, bool overlap_previous);
bool small1d_supported(const frkc2_problem& p, int s);
// 2D FP32 wavefront pass (pass_wf2d.cu): CTAs of WF_NW warps stream column strips of
// 64 WF_NW cells up the grid with up to WF_KMAX stage levels in flight; rows arrive by TMA.
constexpr int WF_NW = 4;
int wf2d_face_pitch(int nx);
// computed / output cell-stages of the wavefront pass at its default launch
double wf2d_recompute(int nx, int ny, int k);
// k stages per pass and s stages per step: every pass (the last may be shorter) needs an
// instantiated stage count (1, 2, 4, 6, 8, 10 or 12)
bool wf2d_supported(const frkc2_problem& p, int k, int s, const void* u);
cudaError_t launch_faces_wf(const frkc2_problem& p, const void* fx, const void* fy, void* out, cudaStream_t st);
// chunk_rows: rows per CTA (0 = one wave of two CTAs per SM); in_real / out_real: the pass reads
// / writes the real state (float [ny][nx]) instead of interleaved (U, V) float2 [ny][nx]
cudaError_t launch_pass_wf2d(const frkc2_problem& p, const PassArgs& a, const void* faces_wf, int chunk_rows,
                             bool in_real, bool out_real, cudaStream_t st, bool overlap_previous,
                             long long wait_limit = 0, int fault_inject = 0);
cudaError_t launch_small1d(const frkc2_problem& p, const frkc2_plan_s& plan, double dt, int nsteps, void* u,
                           const void* fx, unsigned* status, cudaStream_t st, int cluster, int stages_per_exchange,
                           int threads_per_cta);
cudaError_t launch_pass_stream3d(const frkc2_problem& p, const PassArgs& a, cudaStream_t st);
cudaError_t launch_pass_tb2d_df(const frkc2_problem& p, const PassArgs& a, cudaStream_t st, bool overlap_previous);
cudaError_t launch_pass_stream2d_df(const frkc2_problem& p, const PassArgs& a, const void* fen, cudaStream_t st);
cudaError_t launch_pass_paired2d(const frkc2_problem& p, const PassArgs& a, const void* fen, cudaStream_t st);
bool tb2d_supported(const frkc2_problem& p, int k);
size_t generic_smem_bytes(const frkc2_problem& p, const PassArgs& a);
void default_tiles(const frkc2_problem& p, int k, int* tx, int* ty, int* tz);

// One streamed 2D adjoint stage (fixed conductivity).
struct AdjStreamArgs {
  int nx, ny;
  const void* fen;    // face pairs
  const void* W;      // stage state W^l
  int w_complex;      // 0: real array (imaginary part 0), 1: interleaved (U, V)
  const void* L_in;   // lam^{l+1}
  int l_complex;      // 0: real array, 1: interleaved, 2: real part of an interleaved array
  void* L_out;        // lam^l, interleaved
  double* dk;         // dJ/dkappa accumulator or nullptr
  double ca, cb;      // dt a_l / dx^2
};
cudaError_t launch_adj_stream2d(const frkc2_problem& p, const AdjStreamArgs& a, cudaStream_t st);

// Temporally blocked FP32 adjoint (2D fixed conductivity): one pass of nst <= k stages.
struct AdjTbPass {
  int nst;
  // tape pass: forward stages from W^{l0}; out[j] receives W^{l0+1+j} (interleaved), the last
  // as a real array when last_real (the step output)
  const void* in;
  int in_complex;
  void* out[16];
  int last_real;
  // reverse pass: stage j is the j-th from the end; W[j] its tape entry (real when !w_complex)
  const void* W[16];
  int w_complex[16];
  const void* L_in;
  int l_mode;  // 0: real array, 1: interleaved, 2: real part of an interleaved array
  void* L_out;
  double* dk;
  double ca[16], cb[16];  // dt a_l / dx^2 of stage j
};
bool adj_tb2d_supported(const frkc2_problem& p, int k);
cudaError_t launch_tape_tb2d(const frkc2_problem& p, int k, const AdjTbPass& t, const void* fx, const void* fy,
                             unsigned* status, cudaStream_t st);
cudaError_t launch_adjrev_tb2d(const frkc2_problem& p, int k, const AdjTbPass& t, const void* fx, const void* fy,
                               unsigned* status, cudaStream_t st);

void count_launch(int n = 1);

// SM count and resident CTAs per SM of a kernel (at least 1).  Launchers keep the result in a
// function-local static, initialised once and thread-safely on the first call -- which must
// not be inside a stream capture; the library assumes one GPU model per process.
struct Residency {
  cudaError_t err;
  int sms;
  int per_sm;
};
template <class K>
Residency query_residency(K kern, int threads, size_t smem) {
  Residency r{cudaSuccess, 0, 0};
  int dev = 0;
  r.err = cudaGetDevice(&dev);
  if (r.err == cudaSuccess) r.err = cudaDeviceGetAttribute(&r.sms, cudaDevAttrMultiProcessorCount, dev);
  if (r.err == cudaSuccess) r.err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r.per_sm, kern, threads, smem);
  if (r.per_sm < 1) r.per_sm = 1;
  return r;
}

}  // namespace frkc2
