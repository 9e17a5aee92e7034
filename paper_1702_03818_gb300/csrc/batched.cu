// Batched forward step: many independent 2D problems advanced by ONE persistent launch.
//
// Each problem i has its own grid (nx, ny), conductivity field, stage order (plan, s_i),
// dt_i and step count; stages are grouped into passes of k (the pass of Sec. 3, Eq. 13
// applied k times in shared memory, as in the generic tile kernel).  Problem i needs
// T_i = nsteps_i * ceil(s_i / k) passes of N_i tiles.  The work list is a sequence of
// rounds: round r holds, for every problem with T_i > r, all N_i tiles of its pass r
// (problems sorted by T_i, largest first, so the active problems of a round are a prefix).
// CTAs take items in list order from an atomic ticket; an item of pass r waits until the
// problem's completion counter shows all N_i tiles of pass r-1 done (which also means every
// read of the buffer that pass r overwrites is finished).  Every item a CTA waits for was
// taken earlier by a running CTA that does not wait on anything later, so the waits end;
// each wait is still bounded (polls counted) and on expiry the launch latches
// FRKC2_ETIMEOUT in the status word, raises an abort word and every CTA returns.
//
// State buffers are rewritten by other CTAs within the launch, so state loads bypass L1
// (ld.global.cg); a finished tile is published with a device-scope fence before its counter
// increment.  FP32 items run the register-tiled 64 x 64 region of the single-problem FP32
// pass (tb2d_region.cuh: tile 64 - 2k, k-cell recomputed halo), DFLOAT items the float-pair
// region of the single-problem DFLOAT pass (tb2d_df_region.cuh) or, with one stage per pass,
// a float-pair streaming body; each region is a call of its own, not inlined into the item
// loop, so that it keeps the register budget it has in the single-problem pass.  FP64 and MIXED items with one
// stage per pass (the default) run the streaming body of the single-problem pass on a tile of
// 31 columns and a block of rows split among the CTA's warps -- interleaved complex state,
// face pairs, every neighbour difference formed once: 16 FP64 instructions per cell-stage;
// with k > 1 (or kernel 1) they run a k-stage shared-memory tile pass.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <numeric>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "frkc2.h"
#include "frkc2_internal.h"
#include "tb2d_df_region.cuh"
#include "tb2d_region.cuh"

namespace frkc2 {

frkc2_status validate_problem(const frkc2_problem* p);

namespace {

constexpr int BT_THREADS = 256;
constexpr long long DEFAULT_WAIT_LIMIT = 1ll << 22;

struct BProb {
  int nx, ny;
  int tiles_x, ntiles;   // tiles per row of tiles; work items per pass
  int tiles_total;       // tiles per pass (an FP32 item covers up to `group` consecutive tiles)
  int s, passes_per_step, total_passes, extra_copy;
  const void* fx;
  const void* fy;
  const void* fen;     // face pairs (east, north) [ny + 1][nx + 1] for the streaming items
  void* u;
  void* ua;
  void* va;
  void* ub;
  void* vb;
  const double* coef;  // (ca, cb) per stage, dt a_l / dx^2
};

struct BHeader {
  int nprob, nrounds, bc, tx, ty, k, fault_inject;
  int stream_rows;               // > 0: FP64 / MIXED streaming items of 31 columns x this many rows
  int group;                     // FP32: consecutive tiles of one pass per work item
  long long total_items;
  long long wait_limit;
  const BProb* probs;            // sorted by total passes, largest first
  const long long* round_off;    // nrounds + 1 item offsets
  const long long* cum_tiles;    // nprob + 1 tile prefix sums (sorted order)
  unsigned* status;
  unsigned long long* ticket;
  unsigned* abort_flag;
  unsigned* done;                // per problem: tiles completed
};

__device__ __forceinline__ int wrap_b(int g, int n) {
  int r = g % n;
  return r < 0 ? r + n : r;
}

template <class S>
__device__ __forceinline__ S load_cg(const S* p) {
  return __ldcg(p);
}

// state set read by pass r (r >= 1 reads A for odd r, B for even r; pass 0 reads u)
__device__ __forceinline__ void pass_buffers(const BProb& P, int r, const void*& Uin, const void*& Vin,
                                             void*& Uout, void*& Vout, int& l0, int& kq, int k) {
  const int last = P.total_passes + P.extra_copy - 1;
  if (r < P.total_passes) {
    const int q = r % P.passes_per_step;
    l0 = q * k;
    kq = min(k, P.s - l0);
    Uin = r == 0 ? P.u : ((r & 1) ? P.ua : P.ub);
    Vin = (r == 0 || q == 0) ? nullptr : ((r & 1) ? P.va : P.vb);
    const bool step_end = q == P.passes_per_step - 1;
    if (r == last) {
      Uout = P.u;
      Vout = nullptr;
    } else {
      Uout = ((r + 1) & 1) ? P.ua : P.ub;
      Vout = step_end ? nullptr : (((r + 1) & 1) ? P.va : P.vb);
    }
  } else {  // the copy pass of a problem with a single pass: A -> u
    l0 = 0;
    kq = 0;
    Uin = P.ua;
    Vin = nullptr;
    Uout = P.u;
    Vout = nullptr;
  }
}

constexpr int BS_COLS = 31;  // output columns of a streaming item (lane 0 is the west halo)

template <class T> struct BVec2;
template <> struct BVec2<double> { using type = double2; };
template <> struct BVec2<float> { using type = float2; };

// One stage (one pass of k = 1) of a streaming item: column chunk cw (output columns
// 31 cw .. 31 cw + 30, lane 0 reading the column to their west), rows [r0, r1) split evenly
// among the warps, each warp walking up its rows with the south difference and face carried
// in registers and east / west differences shared by shuffles (the single-problem streaming
// pass's arithmetic).  The state comes interleaved (in_real: the real part only) and goes out
// interleaved (out_real: the real part only); state loads go through L2 (other CTAs of the
// launch wrote them).  Returns true if a stored real part is not finite (out_real only).
template <class S, class A, bool PERIODIC>
__device__ __forceinline__ bool stream_item(const BProb& P, int cw, int r0, int r1, const void* in, bool in_real,
                                            void* out, bool out_real, S ca, S cb) {
  using S2 = typename BVec2<S>::type;
  using A2 = typename BVec2<A>::type;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = BT_THREADS / 32;
  const int nx = P.nx, ny = P.ny;
  const int per = (r1 - r0 + nwarps - 1) / nwarps;
  const int y0 = r0 + warp * per, y1 = min(y0 + per, r1);
  bool bad = false;
  if (y0 >= y1) return false;  // warp-uniform
  const A2* __restrict__ FEN = static_cast<const A2*>(P.fen);
  const S* Ur = static_cast<const S*>(in);
  const S2* Wi = static_cast<const S2*>(in);
  S* Uo = static_cast<S*>(out);
  S2* Wo = static_cast<S2*>(out);
  const int x = cw * BS_COLS + lane - 1;
  int xr, xeast;
  bool xin, eastin;
  if (PERIODIC) {
    xr = x < 0 ? x + nx : (x >= nx ? x - nx : x);
    xin = true;
    xeast = xr + 1 == nx ? 0 : xr + 1;
    eastin = true;
  } else {
    xr = x;
    xin = x >= 0 && x < nx;
    xeast = x + 1;
    eastin = xeast >= 0 && xeast < nx;
  }
  const bool has_faces = PERIODIC || (x >= -1 && x < nx);
  const int fcol = (PERIODIC ? xr : x) + 1;
  const bool out_ok = lane >= 1 && x >= 0 && x < nx;
  auto load = [&](int yy, int xx, bool inx) -> S2 {
    S2 w;
    w.x = S(0);
    w.y = S(0);
    int yw = yy;
    if (PERIODIC) {
      if (yw < 0) yw += ny;
      while (yw >= ny) yw -= ny;
    } else if (!(inx && yy >= 0 && yy < ny)) {
      return w;
    }
    const size_t g = size_t(yw) * nx + xx;
    if (in_real)
      w.x = __ldcg(Ur + g);
    else
      w = __ldcg(Wi + g);
    return w;
  };
  auto faces = [&](int yy) -> A2 {
    A2 f;
    f.x = A(0);
    f.y = A(0);
    if (PERIODIC) {
      if (yy < 0) yy += ny;
      while (yy >= ny) yy -= ny;
    } else if (yy >= ny) {
      return f;
    }
    if (!has_faces) return f;
    return __ldg(FEN + size_t(yy + 1) * (nx + 1) + fcol);
  };
  S2 Wc = load(y0, xr, xin);
  A dSU, dSV, ks;
  {
    const S2 Ws = load(y0 - 1, xr, xin);
    ks = faces(y0 - 1).y;
    dSU = A(Wc.x - Ws.x);
    dSV = A(Wc.y - Ws.y);
  }
  S2 Wn = load(y0 + 1, xr, xin);
  A2 f = faces(y0);
  S2 Wen = lane == 31 ? load(y0, xeast, eastin) : Wc;
  for (int y = y0; y < y1; ++y) {
    const S2 Wnn = load(y + 2, xr, xin);
    const A2 fnext = faces(y + 1);
    const S2 Wenn = lane == 31 ? load(y + 1, xeast, eastin) : Wn;
    S Ue = __shfl_down_sync(0xffffffffu, Wc.x, 1);
    S Ve = __shfl_down_sync(0xffffffffu, Wc.y, 1);
    if (lane == 31) {
      Ue = Wen.x;
      Ve = Wen.y;
    }
    const A dEU = A(Ue - Wc.x), dEV = A(Ve - Wc.y);
    const A dNU = A(Wn.x - Wc.x), dNV = A(Wn.y - Wc.y);
    const A dWU = __shfl_up_sync(0xffffffffu, dEU, 1);
    const A dWV = __shfl_up_sync(0xffffffffu, dEV, 1);
    const A kw = __shfl_up_sync(0xffffffffu, f.x, 1);
    const A fU = f.y * dNU - ks * dSU - kw * dWU + f.x * dEU;
    const A fV = f.y * dNV - ks * dSV - kw * dWV + f.x * dEV;
    const S un = Wc.x + ca * S(fU) - cb * S(fV);
    const S vn = Wc.y + ca * S(fV) + cb * S(fU);
    if (out_ok) {
      const size_t g = size_t(y) * nx + x;
      if (out_real) {
        Uo[g] = un;
        bad |= !isfinite(double(un));
      } else {
        S2 w;
        w.x = un;
        w.y = vn;
        Wo[g] = w;
      }
    }
    dSU = dNU;
    dSV = dNV;
    ks = f.y;
    Wc = Wn;
    Wn = Wnn;
    f = fnext;
    Wen = Wenn;
  }
  return bad;
}

// The kernel instantiations of DFLOAT batches (the state is the float pair below): one for the
// register-tiled region items, one for the streaming items (their register budgets differ).
template <bool PERIODIC>
struct DFloatRegions {};
struct DFloatStream {};
template <class S> struct is_df_regions : std::false_type {};
template <bool P> struct is_df_regions<DFloatRegions<P>> : std::true_type {
  static constexpr bool periodic = P;
};

// (h, l) + d as a renormalised float pair (Knuth's TwoSum, then a fast renormalisation)
__device__ __forceinline__ void bdf_add(float& h, float& l, float d) {
  const float s = h + d;
  const float bb = s - h;
  const float e = (h - (s - bb)) + (d - bb);
  const float t = l + e;
  const float hi = s + t;
  l = t - (hi - s);
  h = hi;
}

// One stage of a DFLOAT streaming item: the layout of stream_item with the state as float
// pairs, (U hi, U lo, V hi, V lo) in one float4 a cell, float faces and float arithmetic
// (the single-problem DFLOAT pass's stage).  IN_REAL: the step's first stage, reading the
// double real state and splitting it; OUT_REAL: its last, writing hi + lo as a double (template
// arguments, so the stages between hold no double arithmetic).
template <bool PERIODIC, bool IN_REAL, bool OUT_REAL>
__device__ __forceinline__ bool stream_item_df(const BProb& P, int cw, int r0, int r1, const void* in, void* out,
                                               float ca, float cb) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = BT_THREADS / 32;
  const int nx = P.nx, ny = P.ny;
  const int per = (r1 - r0 + nwarps - 1) / nwarps;
  const int y0 = r0 + warp * per, y1 = min(y0 + per, r1);
  bool bad = false;
  if (y0 >= y1) return false;  // warp-uniform
  const float2* __restrict__ FEN = static_cast<const float2*>(P.fen);
  const double* Ur = static_cast<const double*>(in);
  const float4* Wi = static_cast<const float4*>(in);
  double* Uo = static_cast<double*>(out);
  float4* Wo = static_cast<float4*>(out);
  const int x = cw * BS_COLS + lane - 1;
  int xr, xeast;
  bool xin, eastin;
  if (PERIODIC) {
    xr = x < 0 ? x + nx : (x >= nx ? x - nx : x);
    xin = true;
    xeast = xr + 1 == nx ? 0 : xr + 1;
    eastin = true;
  } else {
    xr = x;
    xin = x >= 0 && x < nx;
    xeast = x + 1;
    eastin = xeast >= 0 && xeast < nx;
  }
  const bool has_faces = PERIODIC || (x >= -1 && x < nx);
  const int fcol = (PERIODIC ? xr : x) + 1;
  const bool out_ok = lane >= 1 && x >= 0 && x < nx;
  auto load = [&](int yy, int xx, bool inx) -> float4 {
    int yw = yy;
    if (PERIODIC) {
      if (yw < 0) yw += ny;
      while (yw >= ny) yw -= ny;
    } else if (!(inx && yy >= 0 && yy < ny)) {
      return make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const size_t g = size_t(yw) * nx + xx;
    if (IN_REAL) {
      const double u = __ldcg(Ur + g);
      const float hi = __double2float_rn(u);
      return make_float4(hi, __double2float_rn(u - double(hi)), 0.f, 0.f);
    }
    return __ldcg(Wi + g);
  };
  auto faces = [&](int yy) -> float2 {
    if (PERIODIC) {
      if (yy < 0) yy += ny;
      while (yy >= ny) yy -= ny;
    } else if (yy >= ny) {
      return make_float2(0.f, 0.f);
    }
    if (!has_faces) return make_float2(0.f, 0.f);
    return __ldg(FEN + size_t(yy + 1) * (nx + 1) + fcol);
  };
  auto diff = [](float ah, float al, float bh, float bl) -> float { return (ah - bh) + (al - bl); };
  float4 Wc = load(y0, xr, xin);
  float dSU, dSV, ks;
  {
    const float4 Ws = load(y0 - 1, xr, xin);
    ks = faces(y0 - 1).y;
    dSU = diff(Wc.x, Wc.y, Ws.x, Ws.y);
    dSV = diff(Wc.z, Wc.w, Ws.z, Ws.w);
  }
  float4 Wn = load(y0 + 1, xr, xin);
  float2 f = faces(y0);
  float4 Wen = lane == 31 ? load(y0, xeast, eastin) : Wc;
  for (int y = y0; y < y1; ++y) {
    const float4 Wnn = load(y + 2, xr, xin);
    const float2 fnext = faces(y + 1);
    const float4 Wenn = lane == 31 ? load(y + 1, xeast, eastin) : Wn;
    float4 We;
    We.x = __shfl_down_sync(0xffffffffu, Wc.x, 1);
    We.y = __shfl_down_sync(0xffffffffu, Wc.y, 1);
    We.z = __shfl_down_sync(0xffffffffu, Wc.z, 1);
    We.w = __shfl_down_sync(0xffffffffu, Wc.w, 1);
    if (lane == 31) We = Wen;
    const float dEU = diff(We.x, We.y, Wc.x, Wc.y), dEV = diff(We.z, We.w, Wc.z, Wc.w);
    const float dNU = diff(Wn.x, Wn.y, Wc.x, Wc.y), dNV = diff(Wn.z, Wn.w, Wc.z, Wc.w);
    const float dWU = __shfl_up_sync(0xffffffffu, dEU, 1);
    const float dWV = __shfl_up_sync(0xffffffffu, dEV, 1);
    const float kw = __shfl_up_sync(0xffffffffu, f.x, 1);
    const float fU = f.y * dNU - ks * dSU - kw * dWU + f.x * dEU;
    const float fV = f.y * dNV - ks * dSV - kw * dWV + f.x * dEV;
    float uh = Wc.x, ul = Wc.y, vh = Wc.z, vl = Wc.w;
    bdf_add(uh, ul, ca * fU - cb * fV);
    bdf_add(vh, vl, ca * fV + cb * fU);
    if (out_ok) {
      const size_t g = size_t(y) * nx + x;
      if (OUT_REAL) {
        const double un = double(uh) + double(ul);
        Uo[g] = un;
        bad |= (__double2hiint(un) & 0x7ff00000) == 0x7ff00000;
      } else {
        Wo[g] = make_float4(uh, ul, vh, vl);
      }
    }
    dSU = dNU;
    dSV = dNV;
    ks = f.y;
    Wc = Wn;
    Wn = Wnn;
    f = fnext;
    Wen = Wenn;
  }
  return bad;
}

// One DFLOAT region as a call of its own (not inlined), so that each of its variants gets the
// register budget it has in the single-problem pass instead of sharing one with the item loop.
template <bool PERIODIC, bool IN_REAL, bool OUT_REAL>
__device__ __noinline__ bool df_region_call(DfShared& sh, int nx, int ny, int k, int kq, int x0, int y0,
                                            const void* in, void* out, const float* FX, const float* FY,
                                            const double* cf) {
  auto coef = [&](int j, float& ca, float& cb) {
    ca = float(cf[2 * j]);
    cb = float(cf[2 * j + 1]);
  };
  return tb2d_df_region<PERIODIC, IN_REAL, OUT_REAL, true>(sh, nx, ny, k, kq, x0, y0, in, out, FX, FY, coef, true,
                                                          [] {});
}

// One FP32 region as a call of its own (not inlined), for the same reason.
template <bool PERIODIC>
__device__ __noinline__ bool fp32_region_call(RegionShared& sh, int nx, int ny, int k, int kq, int x0, int y0,
                                              const float* Uin, const float* Vin, float* Uout, float* Vout,
                                              const float* FX, const float* FY, const double* cf) {
  auto coef = [&](int j, float& ca, float& cb) {
    ca = float(cf[2 * j]);
    cb = float(cf[2 * j + 1]);
  };
  return tb2d_region<PERIODIC, true>(sh, nx, ny, k, kq, x0, y0, Uin, Vin, Uout, Vout, FX, FY, coef, Vout == nullptr);
}

// FP32 items hold a 4 x 4 block of cells per thread in registers: two CTAs per SM
template <class S, class A>
constexpr int bt_min_blocks() {
  return (std::is_same<S, float>::value && std::is_same<A, float>::value) || is_df_regions<S>::value ? 2 : 1;
}

template <class S, class A>
__global__ void __launch_bounds__(BT_THREADS, bt_min_blocks<S, A>()) k_batched(const BHeader h) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long s_item;
  __shared__ int s_prob, s_tile, s_round, s_ok;
  const int tid = threadIdx.x;
  const bool periodic = h.bc == FRKC2_BC_PERIODIC;
  // thread 0 takes the next ticket while the current item computes, so the atomic's round trip
  // is off the path between items (an item still waits only for items of smaller tickets, all
  // taken by running CTAs: the smallest unfinished ticket is always being computed)
  unsigned long long next_ticket = 0;
  bool have_next = false;
  while (true) {
    if (tid == 0) {
      s_item = have_next ? (long long)next_ticket : (long long)atomicAdd(h.ticket, 1ull);
      have_next = false;
      s_ok = 1;
      if (s_item < h.total_items && !*((volatile unsigned*)h.abort_flag)) {
        // decode (round, problem, tile)
        int lo = 0, hi = h.nrounds;  // largest r with round_off[r] <= item
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (h.round_off[mid] <= s_item) lo = mid; else hi = mid;
        }
        const long long rem = s_item - h.round_off[lo];
        int plo = 0, phi = h.nprob;
        while (phi - plo > 1) {
          const int mid = (plo + phi) >> 1;
          if (h.cum_tiles[mid] <= rem) plo = mid; else phi = mid;
        }
        s_round = lo;
        s_prob = plo;
        s_tile = int(rem - h.cum_tiles[plo]);
        // wait for the previous pass of this problem
        const BProb& P = h.probs[plo];
        unsigned need = unsigned(lo) * unsigned(P.ntiles);
        if (h.fault_inject && lo > 0) need = 0xffffffffu;  // a target nothing reaches
        if (lo > 0) {
          long long polls = 0;
          while (*((volatile unsigned*)&h.done[plo]) < need) {
            if (*((volatile unsigned*)h.abort_flag) || ++polls > h.wait_limit) {
              atomicOr(h.status, ST_TIMEOUT);
              atomicExch(h.abort_flag, 1u);
              s_ok = 0;
              break;
            }
            __nanosleep(64);
          }
          __threadfence();
        }
      } else {
        s_ok = 0;
        s_item = h.total_items;
      }
    }
    __syncthreads();
    if (s_item >= h.total_items || !s_ok) break;
    if (tid == 0) {
      next_ticket = atomicAdd(h.ticket, 1ull);
      have_next = true;
    }
    const BProb& P = h.probs[s_prob];
    const void* Uin_v;
    const void* Vin_v;
    void* Uout_v;
    void* Vout_v;
    int l0, kq;
    pass_buffers(P, s_round, Uin_v, Vin_v, Uout_v, Vout_v, l0, kq, h.k);
    const int tyi = s_tile / P.tiles_x, txi = s_tile - tyi * P.tiles_x;
    if constexpr (is_df_regions<S>::value) {
      // DFLOAT float-pair register-tiled regions of k stages: real input at a step's first
      // pass, real output at its last
      constexpr bool PER = is_df_regions<S>::periodic;
      const int q = s_round < P.total_passes ? s_round % P.passes_per_step : 0;
      const bool in_real = q == 0, out_real = q == P.passes_per_step - 1;
      bool bad = false;
      DfShared& dsh = *reinterpret_cast<DfShared*>(smem);
      const double* cf = P.coef + 2 * l0;
      const float* FXp = static_cast<const float*>(P.fx);
      const float* FYp = static_cast<const float*>(P.fy);
      for (int g = 0; g < h.group; ++g) {
        const int tile = s_tile * h.group + g;
        if (tile >= P.tiles_total) break;  // block-uniform
        const int ty_i = tile / P.tiles_x, tx_i = tile - ty_i * P.tiles_x;
        const int x0 = tx_i * h.tx - h.k, y0 = ty_i * h.ty - h.k;
        auto region = [&](auto inr, auto outr) {
          return df_region_call<PER, decltype(inr)::value, decltype(outr)::value>(dsh, P.nx, P.ny, h.k, kq, x0, y0,
                                                                                  Uin_v, Uout_v, FXp, FYp, cf);
        };
        using T_ = std::true_type;
        using F_ = std::false_type;
        bad |= in_real ? (out_real ? region(T_{}, T_{}) : region(T_{}, F_{}))
                       : (out_real ? region(F_{}, T_{}) : region(F_{}, F_{}));
        __syncthreads();  // the region's shared buffers are reused by the next tile
      }
      if (bad) atomicOr(h.status, ST_NONFINITE);
    } else if constexpr (std::is_same<S, DFloatStream>::value) {
      // DFLOAT streaming items of one stage
      const int q = s_round < P.total_passes ? s_round % P.passes_per_step : 0;
      const bool in_real = q == 0, out_real = q == P.passes_per_step - 1;
      bool bad = false;
      const float ca = float(P.coef[2 * l0]), cb = float(P.coef[2 * l0 + 1]);
      const int r0 = tyi * h.stream_rows, r1 = min(r0 + h.stream_rows, P.ny);
      if (periodic) {
        if (in_real && out_real)
          bad = stream_item_df<true, true, true>(P, txi, r0, r1, Uin_v, Uout_v, ca, cb);
        else if (in_real)
          bad = stream_item_df<true, true, false>(P, txi, r0, r1, Uin_v, Uout_v, ca, cb);
        else if (out_real)
          bad = stream_item_df<true, false, true>(P, txi, r0, r1, Uin_v, Uout_v, ca, cb);
        else
          bad = stream_item_df<true, false, false>(P, txi, r0, r1, Uin_v, Uout_v, ca, cb);
      } else {
        if (in_real && out_real)
          bad = stream_item_df<false, true, true>(P, txi, r0, r1, Uin_v, Uout_v, ca, cb);
        else if (in_real)
          bad = stream_item_df<false, true, false>(P, txi, r0, r1, Uin_v, Uout_v, ca, cb);
        else if (out_real)
          bad = stream_item_df<false, false, true>(P, txi, r0, r1, Uin_v, Uout_v, ca, cb);
        else
          bad = stream_item_df<false, false, false>(P, txi, r0, r1, Uin_v, Uout_v, ca, cb);
      }
      if (bad) atomicOr(h.status, ST_NONFINITE);
    } else if constexpr (std::is_same<S, float>::value && std::is_same<A, float>::value) {
      __shared__ RegionShared rsh;
      const float* Uin = static_cast<const float*>(Uin_v);
      const float* Vin = static_cast<const float*>(Vin_v);
      float* Uout = static_cast<float*>(Uout_v);
      float* Vout = static_cast<float*>(Vout_v);
      bool bad = false;
      // the item's tiles: consecutive tiles of the pass, one region after another
      for (int g = 0; g < h.group; ++g) {
        const int tile = s_tile * h.group + g;
        if (tile >= P.tiles_total) break;  // block-uniform
        const int ty_i = tile / P.tiles_x, tx_i = tile - ty_i * P.tiles_x;
        const int x0 = tx_i * h.tx - h.k, y0 = ty_i * h.ty - h.k;
        bad |= periodic ? fp32_region_call<true>(rsh, P.nx, P.ny, h.k, kq, x0, y0, Uin, Vin, Uout, Vout,
                                                 static_cast<const float*>(P.fx), static_cast<const float*>(P.fy),
                                                 P.coef + 2 * l0)
                        : fp32_region_call<false>(rsh, P.nx, P.ny, h.k, kq, x0, y0, Uin, Vin, Uout, Vout,
                                                  static_cast<const float*>(P.fx), static_cast<const float*>(P.fy),
                                                  P.coef + 2 * l0);
        __syncthreads();  // the region's shared exchange buffers are reused by the next tile
      }
      if (bad) atomicOr(h.status, ST_NONFINITE);
    } else if (h.stream_rows > 0) {
      // one stage: real input at a step's first stage, real output at its last
      const int q = s_round < P.total_passes ? s_round % P.passes_per_step : 0;
      const S ca = S(P.coef[2 * l0]), cb = S(P.coef[2 * l0 + 1]);
      const int r0 = tyi * h.stream_rows, r1 = min(r0 + h.stream_rows, P.ny);
      const bool in_real = q == 0, out_real = q == P.passes_per_step - 1;
      const bool bad = periodic ? stream_item<S, A, true>(P, txi, r0, r1, Uin_v, in_real, Uout_v, out_real, ca, cb)
                                : stream_item<S, A, false>(P, txi, r0, r1, Uin_v, in_real, Uout_v, out_real, ca, cb);
      if (bad) atomicOr(h.status, ST_NONFINITE);
    } else {
      const S* Uin = static_cast<const S*>(Uin_v);
      const S* Vin = static_cast<const S*>(Vin_v);
      const A* FX = static_cast<const A*>(P.fx);
      const A* FY = static_cast<const A*>(P.fy);
      const int nx = P.nx, ny = P.ny;
      const int RX = h.tx + 2 * kq, RY = h.ty + 2 * kq, R = RX * RY;
      S* ub0 = reinterpret_cast<S*>(smem);
      S* vb0 = ub0 + R;
      S* ub1 = vb0 + R;
      S* vb1 = ub1 + R;
      A* fxs = reinterpret_cast<A*>(vb1 + R);
      A* fys = fxs + R;
      const int x0 = txi * h.tx - kq, y0 = tyi * h.ty - kq;
      for (int idx = tid; idx < R; idx += BT_THREADS) {
        const int y = idx / RX, x = idx - y * RX;
        const int gx = x0 + x, gy = y0 + y;
        S uu = S(0), vv = S(0);
        A a0 = A(0), a1 = A(0);
        if (periodic) {
          const int wx = wrap_b(gx, nx), wy = wrap_b(gy, ny);
          const size_t g = size_t(wy) * nx + wx;
          uu = load_cg(Uin + g);
          if (Vin) vv = load_cg(Vin + g);
          a0 = FX[size_t(wy) * (nx + 1) + wx];
          a1 = FY[size_t(wy) * nx + wx];
        } else {
          const bool inx = gx >= 0 && gx < nx, iny = gy >= 0 && gy < ny;
          if (inx && iny) {
            const size_t g = size_t(gy) * nx + gx;
            uu = load_cg(Uin + g);
            if (Vin) vv = load_cg(Vin + g);
          }
          if (iny && gx >= 0 && gx <= nx) a0 = FX[size_t(gy) * (nx + 1) + gx];
          if (inx && gy >= 0 && gy <= ny) a1 = FY[size_t(gy) * nx + gx];
        }
        ub0[idx] = uu;
        vb0[idx] = vv;
        ub1[idx] = S(0);
        vb1[idx] = S(0);
        fxs[idx] = a0;
        fys[idx] = a1;
      }
      __syncthreads();
      for (int j = 1; j <= kq; ++j) {
        const S* us = (j & 1) ? ub0 : ub1;
        const S* vs = (j & 1) ? vb0 : vb1;
        S* ud = (j & 1) ? ub1 : ub0;
        S* vd = (j & 1) ? vb1 : vb0;
        const S ca = S(P.coef[2 * (l0 + j - 1)]), cb = S(P.coef[2 * (l0 + j - 1) + 1]);
        const int w = RX - 2 * j, hgt = RY - 2 * j;
        for (int idx = tid; idx < w * hgt; idx += BT_THREADS) {
          const int y = j + idx / w, x = j + idx % w;
          const int i = y * RX + x;
          if (!periodic) {
            const int gx = x0 + x, gy = y0 + y;
            if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) {
              ud[i] = S(0);
              vd[i] = S(0);
              continue;
            }
          }
          const S Uc = us[i], Vc = vs[i];
          const A fe = fxs[i + 1], fw = fxs[i], fn = fys[i + RX], fs = fys[i];
          const A fR = fe * A(us[i + 1] - Uc) + fw * A(us[i - 1] - Uc) + fn * A(us[i + RX] - Uc) +
                       fs * A(us[i - RX] - Uc);
          const A fI = fe * A(vs[i + 1] - Vc) + fw * A(vs[i - 1] - Vc) + fn * A(vs[i + RX] - Vc) +
                       fs * A(vs[i - RX] - Vc);
          ud[i] = Uc + ca * S(fR) - cb * S(fI);
          vd[i] = Vc + ca * S(fI) + cb * S(fR);
        }
        __syncthreads();
      }
      const S* uf = (kq & 1) ? ub1 : ub0;
      const S* vf = (kq & 1) ? vb1 : vb0;
      S* Uout = static_cast<S*>(Uout_v);
      S* Vout = static_cast<S*>(Vout_v);
      const int ox = txi * h.tx, oy = tyi * h.ty;
      const int ex = min(h.tx, nx - ox), ey = min(h.ty, ny - oy);
      bool bad = false;
      for (int idx = tid; idx < ex * ey; idx += BT_THREADS) {
        const int y = idx / ex, x = idx - y * ex;
        const int i = (y + kq) * RX + (x + kq);
        const size_t g = size_t(oy + y) * nx + (ox + x);
        const S uu = uf[i];
        Uout[g] = uu;
        if (Vout) Vout[g] = vf[i];
        if (!Vout && !isfinite(double(uu))) bad = true;
      }
      if (bad) atomicOr(h.status, ST_NONFINITE);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) atomicAdd(&h.done[s_prob], 1u);
  }
}

struct LaunchCfg {
  int precision;
  bool df_stream;  // DFLOAT streaming items (else DFLOAT region items)
  bool periodic;
  size_t smem;
  int grid;
  void* counters;
  size_t counter_bytes;
  BHeader header;
};

std::mutex g_mu;
std::unordered_map<void*, LaunchCfg> g_cfg;

struct BatchPlanHost {
  std::vector<int> order;         // sorted problem indices
  std::vector<BProb> probs;       // sorted
  std::vector<long long> round_off, cum_tiles;
  std::vector<double> coef;       // all problems' (ca, cb)
  std::vector<size_t> coef_off;   // per sorted problem, in doubles
  size_t off_hdr, off_probs, off_round, off_cum, off_coef, off_counters, off_faces, off_states, total;
  size_t counter_bytes;
  int nrounds;
  long long total_items;
};

// FP32 and DFLOAT region items: consecutive 64 x 64 regions of one pass per work item
// (tune->tile_z; default 4),
// which spreads the per-item hand-over (ticket, decode, dependency check, completion fence)
// over several regions
int batch_group(int precision, const frkc2_tuning* tune, bool streaming) {
  if (streaming || (precision != FRKC2_FP32 && precision != FRKC2_DFLOAT)) return 1;
  return (tune && tune->tile_z) ? tune->tile_z : 4;
}

// FP64 / MIXED batches with one stage per pass run streaming items unless kernel 1 (the shared-
// memory tile pass) is asked for
bool batch_streaming(int precision, int k, const frkc2_tuning* tune) {
  return precision != FRKC2_FP32 && k == 1 && !(tune && tune->kernel == 1);
}

// dynamic shared memory of an item: none for the FP32 register-tiled regions and the streaming
// items, the k-halo tile of state ping-pong buffers and face conductivities otherwise
size_t batch_smem(int precision, int tx, int ty, int k, bool streaming = false) {
  if (precision == FRKC2_FP32 || streaming) return 0;
  if (precision == FRKC2_DFLOAT) return sizeof(DfShared);  // the float-pair regions
  return size_t(tx + 2 * k) * (ty + 2 * k) * (4 * state_bytes(precision) + 2 * arith_bytes(precision));
}

frkc2_status batch_geometry(int nprob, const frkc2_plan_t* plans, const frkc2_problem* probs, const int* nsteps,
                            const frkc2_tuning* tune, int* k_out, int* tx_out, int* ty_out) {
  if (nprob < 1 || !plans || !probs || !nsteps) return FRKC2_EINVAL;
  const frkc2_problem& p0 = probs[0];
  for (int i = 0; i < nprob; ++i) {
    const frkc2_status v = validate_problem(&probs[i]);
    if (v != FRKC2_OK) return v;
    if (!plans[i] || nsteps[i] < 1) return FRKC2_EINVAL;
    if (probs[i].ndim != 2 || probs[i].kappa_kind == FRKC2_KAPPA_POWER) return FRKC2_EUNSUPPORTED;
    if (probs[i].precision != p0.precision || probs[i].bc != p0.bc) return FRKC2_EINVAL;
  }
  const bool regions = p0.precision == FRKC2_FP32 || p0.precision == FRKC2_DFLOAT;
  int k = (tune && tune->k) ? tune->k : (regions ? 8 : 1);
  // DFLOAT items: float-pair regions, or streaming items with one stage per pass; no tile pass
  if (p0.precision == FRKC2_DFLOAT && tune && tune->kernel == 1) return FRKC2_EUNSUPPORTED;
  int tx = (tune && tune->tile_x) ? tune->tile_x : 64;
  int ty = (tune && tune->tile_y) ? tune->tile_y : 16;
  if (k < 1 || k > KMAX || tx < 1 || ty < 1) return FRKC2_EINVAL;
  if (regions && !batch_streaming(p0.precision, k, tune)) {  // register-tiled regions: region minus halo
    if (2 * k >= RT_R) return FRKC2_EINVAL;
    tx = ty = RT_R - 2 * k;
  } else if (batch_streaming(p0.precision, k, tune)) {  // streaming items: 31 columns x a row block
    tx = BS_COLS;
    ty = (tune && tune->tile_y) ? tune->tile_y : 128;
  }
  if (batch_smem(p0.precision, tx, ty, k, batch_streaming(p0.precision, k, tune)) > 200 * 1024) return FRKC2_EINVAL;
  *k_out = k;
  *tx_out = tx;
  *ty_out = ty;
  return FRKC2_OK;
}

frkc2_status batch_plan(int nprob, const frkc2_plan_t* plans, const frkc2_problem* probs, const double* dt,
                        const int* nsteps, const frkc2_tuning* tune, BatchPlanHost& B, int& k, int& tx, int& ty) {
  frkc2_status v = batch_geometry(nprob, plans, probs, nsteps, tune, &k, &tx, &ty);
  if (v != FRKC2_OK) return v;
  const size_t SB = state_bytes(probs[0].precision), AB = arith_bytes(probs[0].precision);
  const int group = batch_group(probs[0].precision, tune, batch_streaming(probs[0].precision, k, tune));
  if (group < 1 || group > 64) return FRKC2_EINVAL;
  std::vector<int> T(nprob);
  for (int i = 0; i < nprob; ++i) {
    const int P = (plans[i]->s + k - 1) / k;
    T[i] = nsteps[i] * P;
  }
  B.order.resize(nprob);
  std::iota(B.order.begin(), B.order.end(), 0);
  std::stable_sort(B.order.begin(), B.order.end(), [&](int a, int b) { return T[a] > T[b]; });
  B.probs.resize(nprob);
  B.cum_tiles.assign(nprob + 1, 0);
  B.coef.clear();
  B.coef_off.resize(nprob);
  for (int r = 0; r < nprob; ++r) {
    const int i = B.order[r];
    const frkc2_problem& p = probs[i];
    BProb& P = B.probs[r];
    P.nx = int(p.n[0]);
    P.ny = int(p.n[1]);
    P.tiles_x = (P.nx + tx - 1) / tx;
    P.tiles_total = P.tiles_x * ((P.ny + ty - 1) / ty);
    P.ntiles = (P.tiles_total + group - 1) / group;
    P.s = plans[i]->s;
    P.passes_per_step = (P.s + k - 1) / k;
    P.total_passes = T[i];
    P.extra_copy = T[i] == 1 ? 1 : 0;
    B.cum_tiles[r + 1] = B.cum_tiles[r] + P.ntiles;
    B.coef_off[r] = B.coef.size();
    const double h2 = p.dx * p.dx;
    if (dt) {
      if (!(dt[i] > 0.0) || !std::isfinite(dt[i])) return FRKC2_EINVAL;
      for (int l = 0; l < P.s; ++l) {
        B.coef.push_back(dt[i] * plans[i]->a_re[l] / h2);
        B.coef.push_back(dt[i] * plans[i]->a_im[l] / h2);
      }
    } else {
      B.coef.resize(B.coef.size() + 2 * size_t(P.s), 0.0);
    }
  }
  const int maxT = B.probs[0].total_passes + B.probs[0].extra_copy;
  B.nrounds = maxT;
  B.round_off.assign(maxT + 1, 0);
  for (int r = 0; r < maxT; ++r) {
    int active = 0;
    while (active < nprob && B.probs[active].total_passes + B.probs[active].extra_copy > r) ++active;
    B.round_off[r + 1] = B.round_off[r] + B.cum_tiles[active];
  }
  B.total_items = B.round_off[maxT];
  // workspace layout
  size_t off = 256;  // status word
  B.off_hdr = off;
  off += 256;
  B.off_probs = off;
  off += align256(sizeof(BProb) * nprob);
  B.off_round = off;
  off += align256(sizeof(long long) * (maxT + 1));
  B.off_cum = off;
  off += align256(sizeof(long long) * (nprob + 1));
  B.off_coef = off;
  off += align256(sizeof(double) * B.coef.size());
  B.off_counters = off;  // ticket (8 B), abort (4 B), done[nprob]
  B.counter_bytes = 16 + sizeof(unsigned) * size_t(nprob);
  off += align256(B.counter_bytes);
  B.off_faces = off;
  const bool streaming = batch_streaming(probs[0].precision, k, tune);
  for (int r = 0; r < nprob; ++r) {
    const BProb& P = B.probs[r];
    off += align256(size_t(P.ny) * (P.nx + 1) * AB) + align256(size_t(P.ny + 1) * P.nx * AB);
    if (streaming) off += align256(size_t(P.ny + 1) * (P.nx + 1) * 2 * AB);  // face pairs
  }
  B.off_states = off;
  for (int r = 0; r < nprob; ++r) {
    const BProb& P = B.probs[r];
    off += 4 * align256(size_t(P.nx) * P.ny * SB);
  }
  B.total = off;
  return FRKC2_OK;
}

int persistent_grid(int precision, size_t smem, bool df_stream) {
  int dev = 0, sms = 152, per = 1;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  if (precision == FRKC2_FP64)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batched<double, double>, BT_THREADS, smem);
  else if (precision == FRKC2_FP32)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batched<float, float>, BT_THREADS, smem);
  else if (precision == FRKC2_DFLOAT && df_stream)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batched<DFloatStream, float>, BT_THREADS, smem);
  else if (precision == FRKC2_DFLOAT)  // the periodic and Dirichlet instantiations share their budget
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batched<DFloatRegions<true>, float>, BT_THREADS, smem);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batched<double, float>, BT_THREADS, smem);
  if (e != cudaSuccess || per < 1) per = 1;
  return sms * per;
}

template <class S, class A>
cudaError_t set_smem(size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(k_batched<S, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
}

}  // namespace
}  // namespace frkc2

using namespace frkc2;

extern "C" {

frkc2_status frkc2_batch_workspace_size(int nprob, const frkc2_plan_t* plans, const frkc2_problem* probs,
                                        const int* nsteps, const frkc2_tuning* tune, size_t* bytes) {
  if (!bytes) return FRKC2_EINVAL;
  BatchPlanHost B;
  int k, tx, ty;
  const frkc2_status v = batch_plan(nprob, plans, probs, nullptr, nsteps, tune, B, k, tx, ty);
  if (v != FRKC2_OK) return v;
  *bytes = B.total;
  return FRKC2_OK;
}

frkc2_status frkc2_batch_prepare(int nprob, const frkc2_plan_t* plans, const frkc2_problem* probs,
                                 const double* dt, const int* nsteps, void* const* u, const frkc2_tuning* tune,
                                 void* ws, size_t ws_bytes, void* stream) {
  if (!dt || !u || !ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return FRKC2_EINVAL;
  BatchPlanHost B;
  int k, tx, ty;
  frkc2_status v = batch_plan(nprob, plans, probs, dt, nsteps, tune, B, k, tx, ty);
  if (v != FRKC2_OK) return v;
  if (ws_bytes < B.total) return FRKC2_ENOMEM;
  for (int i = 0; i < nprob; ++i)
    if (!u[i]) return FRKC2_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(ws);
  const int prec = probs[0].precision;
  const size_t SB = state_bytes(prec), AB = arith_bytes(prec);
  const bool streaming = batch_streaming(prec, k, tune);
  // per-problem pointers and face conductivities
  size_t fo = B.off_faces, so = B.off_states;
  for (int r = 0; r < nprob; ++r) {
    BProb& P = B.probs[r];
    const int i = B.order[r];
    void* fx = base + fo;
    fo += align256(size_t(P.ny) * (P.nx + 1) * AB);
    void* fy = base + fo;
    fo += align256(size_t(P.ny + 1) * P.nx * AB);
    P.fx = fx;
    P.fy = fy;
    P.fen = nullptr;
    if (streaming) {
      void* fen = base + fo;
      fo += align256(size_t(P.ny + 1) * (P.nx + 1) * 2 * AB);
      P.fen = fen;
    }
    const size_t sb = align256(size_t(P.nx) * P.ny * SB);
    P.ua = base + so;
    P.va = base + so + sb;
    P.ub = base + so + 2 * sb;
    P.vb = base + so + 3 * sb;
    so += 4 * sb;
    P.u = u[i];
    P.coef = reinterpret_cast<const double*>(base + B.off_coef) + B.coef_off[r];
    if (launch_faces(probs[i], fx, fy, nullptr, st) != cudaSuccess) return FRKC2_ECUDA;
    if (streaming && launch_face_pairs(probs[i], fx, fy, const_cast<void*>(P.fen), st) != cudaSuccess)
      return FRKC2_ECUDA;
  }
  BHeader h{};
  h.nprob = nprob;
  h.nrounds = B.nrounds;
  h.bc = probs[0].bc;
  h.tx = tx;
  h.ty = ty;
  h.k = k;
  h.stream_rows = streaming ? ty : 0;
  h.group = batch_group(prec, tune, streaming);
  h.fault_inject = tune ? tune->fault_inject : 0;
  h.total_items = B.total_items;
  h.wait_limit = (tune && tune->wait_limit > 0) ? tune->wait_limit : DEFAULT_WAIT_LIMIT;
  h.probs = reinterpret_cast<const BProb*>(base + B.off_probs);
  h.round_off = reinterpret_cast<const long long*>(base + B.off_round);
  h.cum_tiles = reinterpret_cast<const long long*>(base + B.off_cum);
  h.status = reinterpret_cast<unsigned*>(base);
  h.ticket = reinterpret_cast<unsigned long long*>(base + B.off_counters);
  h.abort_flag = reinterpret_cast<unsigned*>(base + B.off_counters + 8);
  h.done = reinterpret_cast<unsigned*>(base + B.off_counters + 16);
  auto up = [&](size_t off, const void* src, size_t n) {
    return n == 0 || cudaMemcpyAsync(base + off, src, n, cudaMemcpyHostToDevice, st) == cudaSuccess;
  };
  if (!up(B.off_probs, B.probs.data(), sizeof(BProb) * nprob) ||
      !up(B.off_round, B.round_off.data(), sizeof(long long) * B.round_off.size()) ||
      !up(B.off_cum, B.cum_tiles.data(), sizeof(long long) * B.cum_tiles.size()) ||
      !up(B.off_coef, B.coef.data(), sizeof(double) * B.coef.size()))
    return FRKC2_ECUDA;
  // the pageable-source copies above are staged before they return; make the uploads
  // complete before the host vectors go out of scope
  if (cudaStreamSynchronize(st) != cudaSuccess) return FRKC2_ECUDA;
  LaunchCfg cfg{};
  cfg.precision = prec;
  cfg.smem = batch_smem(prec, tx, ty, k, streaming);
  cfg.df_stream = prec == FRKC2_DFLOAT && streaming;
  cfg.periodic = probs[0].bc == FRKC2_BC_PERIODIC;
  cudaError_t e;
  if (prec == FRKC2_FP64)
    e = set_smem<double, double>(cfg.smem);
  else if (prec == FRKC2_FP32)
    e = set_smem<float, float>(cfg.smem);
  else if (cfg.df_stream)
    e = set_smem<DFloatStream, float>(cfg.smem);
  else if (prec == FRKC2_DFLOAT)
    e = cfg.periodic ? set_smem<DFloatRegions<true>, float>(cfg.smem) : set_smem<DFloatRegions<false>, float>(cfg.smem);
  else
    e = set_smem<double, float>(cfg.smem);
  if (e != cudaSuccess) return FRKC2_ECUDA;
  cfg.grid = persistent_grid(prec, cfg.smem, cfg.df_stream);
  if (cfg.grid > B.total_items) cfg.grid = int(B.total_items);
  cfg.counters = base + B.off_counters;
  cfg.counter_bytes = B.counter_bytes;
  cfg.header = h;
  std::lock_guard<std::mutex> lk(g_mu);
  g_cfg[ws] = cfg;
  return FRKC2_OK;
}

frkc2_status frkc2_batch_launch(void* ws, void* stream) {
  const frkc2::NvtxRange call_range("frkc2_batch_launch");
  if (!ws) return FRKC2_EINVAL;
  LaunchCfg cfg;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cfg.find(ws);
    if (it == g_cfg.end()) return FRKC2_EINVAL;  // not prepared
    cfg = it->second;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(cfg.counters, 0, cfg.counter_bytes, st) != cudaSuccess) return FRKC2_ECUDA;
  switch (cfg.precision) {
    case FRKC2_FP64: k_batched<double, double><<<cfg.grid, BT_THREADS, cfg.smem, st>>>(cfg.header); break;
    case FRKC2_FP32: k_batched<float, float><<<cfg.grid, BT_THREADS, cfg.smem, st>>>(cfg.header); break;
    case FRKC2_DFLOAT:
      if (cfg.df_stream)
        k_batched<DFloatStream, float><<<cfg.grid, BT_THREADS, cfg.smem, st>>>(cfg.header);
      else if (cfg.periodic)
        k_batched<DFloatRegions<true>, float><<<cfg.grid, BT_THREADS, cfg.smem, st>>>(cfg.header);
      else
        k_batched<DFloatRegions<false>, float><<<cfg.grid, BT_THREADS, cfg.smem, st>>>(cfg.header);
      break;
    default: k_batched<double, float><<<cfg.grid, BT_THREADS, cfg.smem, st>>>(cfg.header); break;
  }
  count_launch();
  return cudaGetLastError() == cudaSuccess ? FRKC2_OK : FRKC2_ECUDA;
}

frkc2_status frkc2_step_batched(int nprob, const frkc2_plan_t* plans, const frkc2_problem* probs, const double* dt,
                                const int* nsteps, void* const* u, const frkc2_tuning* tune, void* ws,
                                size_t ws_bytes, void* stream) {
  const frkc2_status v = frkc2_batch_prepare(nprob, plans, probs, dt, nsteps, u, tune, ws, ws_bytes, stream);
  if (v != FRKC2_OK) return v;
  return frkc2_batch_launch(ws, stream);
}

}  // extern "C"
