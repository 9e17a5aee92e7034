// 2D temporally blocked pass for FP32 (fixed conductivity) as a wavefront along y: k stages of
// Sec. 3, Eq. 13 per HBM round trip, with the recomputed halo confined to the strip edges.
//
// A CTA of NW warps owns a strip of CW = 64 NW columns (two adjacent cells per thread) and a
// chunk of H rows.  It walks up the chunk one row per iteration and keeps every stage level in
// flight: at iteration t, level j (1..kq) applies stage j to row t - j, from level j-1's row
// t - j (computed at iteration t - 1 and kept in registers), its row t - j + 1 (computed a moment
// earlier in the same iteration) and its row t - j - 1 through the south face flux, carried
// in registers from level j's own previous row.  Level kq's row is the pass output.  The valid
// region shrinks by one column per level at each strip edge, and one row per level at the
// chunk start, so the strip recomputes 2h halo columns (h = k rounded up to 4) and the chunk
// k - 1 rows per level: about 1.07 x 1.12 the output cell-stages at k = 8 on 2048^2 (the 64 x 64
// regions of k_tb2d_reg recompute 1.78x).
//
// Rows arrive by TMA: one elected thread issues 1D bulk copies (cp.async.bulk) of row t + L's
// state segment and face segment into a ring of R = kq + L + 1 shared-memory rows, completing
// on the row's mbarrier; every thread waits (bounded) on that mbarrier before reading row t.
// Periodic strips that cross x = 0 or x = nx take two copies.  A cell is an interleaved (U, V)
// float2, so differences, face fluxes and the complex update act on both components at once as
// packed two-lane FP32 instructions (add / mul / fma .f32x2).  Face fluxes are formed once per
// face: a thread's east flux of its second cell is the next thread's west flux (shuffle); the
// north flux of a row is the south flux of the row above (register carry).  Neighbour values
// beyond the warp come through a small shared array written once per iteration by the warps'
// edge lanes (double-buffered by iteration parity, one barrier per iteration).
//
// Per computed cell-stage: 16 FP32 lane operations (as packed and scalar instructions), 2
// shuffles and one 8-byte shared load of face conductivities; HBM per output cell and pass: 8
// bytes of state in, 8 out, 8 of faces.
#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

#include "frkc2_internal.h"

namespace frkc2 {
namespace {

constexpr int WF_RING = 16;  // rows of the shared-memory ring (a power of two)

struct WfArgs {
  int nx, ny;
  int kq;                 // stages in this pass (the kernel's K)
  int h;                  // halo columns per strip side (kq rounded up to a multiple of 4)
  int ow;                 // output columns per strip: CW - 2h
  int H;                  // rows per chunk
  int pitch_f;            // face array pitch in float2 elements
  int in_real, out_real;  // the pass reads / writes the real state instead of interleaved (U, V)
  const void* in;         // real float [ny][nx] or interleaved float2 [ny][nx]
  void* out;
  const float2* faces;    // [ny + 1][pitch_f]: (k_east, k_north) of cell (x, y) at [y + 1][x + 2]
  unsigned* status;
  int check_finite;
  long long wait_limit;   // polls of a bounded mbarrier wait
  float ca[KMAX];         // dt Re(a_l) / dx^2 for the pass's stages, rounded to float once
  float cb[KMAX];
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Waits for the completion of the phase with the given parity; false after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit) {
  for (long long i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 1D bulk copy global -> shared, completing `bytes` on the mbarrier (16-byte aligned addresses
// and a size that is a multiple of 16).
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 scale(float k, float2 d) { return make_float2(k * d.x, k * d.y); }

// Up to two segments of a logical column range [a, a + n) of a row: (first global column,
// length, offset in the range).  Periodic columns wrap (n <= nx + 2); Dirichlet ones are
// clipped to [lo_lim, hi_lim).
struct Segs {
  int g[2], len[2], off[2], n;
};

template <bool PERIODIC>
__device__ __forceinline__ Segs segments(int a, int n, int nx, int lo_lim, int hi_lim) {
  Segs s;
  s.n = 0;
  s.g[0] = s.g[1] = s.len[0] = s.len[1] = s.off[0] = s.off[1] = 0;
  if (PERIODIC) {
    int a0 = a;
    if (a0 < 0) a0 += nx;
    if (a0 >= nx) a0 -= nx;
    if (a0 < 0 || a0 >= nx) a0 = ((a % nx) + nx) % nx;
    const int first = min(n, nx - a0);
    s.g[0] = a0;
    s.len[0] = first;
    s.n = 1;
    if (first < n) {
      s.len[1] = n - first;
      s.off[1] = first;
      s.n = 2;
    }
  } else {
    const int lo = max(a, lo_lim), hi = min(a + n, hi_lim);
    if (hi > lo) {
      s.g[0] = lo;
      s.len[0] = hi - lo;
      s.off[0] = lo - a;
      s.n = 1;
    }
  }
  return s;
}

struct Cells {
  float2 c0, c1;  // (U, V) of the thread's two cells
};

// FAULT (testing only, one instantiation): the chunk's first row is never copied, so every
// thread's bounded wait on it must run out.  A template argument, since even a test outside
// the loop measurably changed the normal kernel.
template <int K, bool PERIODIC, bool FAULT = false>
__global__ void __launch_bounds__(WF_NW * 32, 2) k_wf2d(const WfArgs p) {
  constexpr int NW = WF_NW;
  constexpr int CW = 64 * NW;                       // computed columns of the strip
  constexpr int SB = CW * 8;                        // state bytes of a ring row
  constexpr int ROWB = SB + (CW + 2) * 8;           // + faces of strip columns -2 .. CW - 1
  constexpr int L = WF_RING - K - 1;                // rows the copies run ahead of their use
  constexpr int KE = (K + 1) / 2 * 2;               // edge entries per warp side (even: 16-byte pairs)
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem);                      // WF_RING barriers
  float2* edge = reinterpret_cast<float2*>(smem + 256);                    // [2][NW][2][KE]
  unsigned char* ring = smem + 256 + ((2 * NW * 2 * KE * 8 + 127) / 128) * 128;

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int cx = 2 * tid;                           // strip column of the thread's first cell
  const int nx = p.nx, ny = p.ny;
  const bool in_real = p.in_real, out_real = p.out_real;
  const int xs = blockIdx.x * p.ow - p.h;           // grid column of strip column 0
  const int y0 = blockIdx.y * p.H, y1 = min(y0 + p.H, ny);
  const int t0 = y0 - K, te = y1 - 1 + K;            // first and last iteration (row loaded)

  // the row copies are the same for every row of the CTA but for the row offset: the strip's
  // state segment(s) and face segment(s) (one thread issues them)
  const int es = in_real ? 4 : 8;
  Segs ss = segments<PERIODIC>(xs, CW, nx, 0, nx);
  Segs fs = segments<PERIODIC>(xs - 2, CW + 2, nx, -2, nx);
  uint32_t sbytes = 0, fbytes = 0;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    sbytes += uint32_t(ss.len[i]) * es;
    fbytes += uint32_t(fs.len[i]) * 8;
  }

  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (tid == 0) {
#pragma unroll
    for (int i = 0; i < WF_RING; ++i) mbar_init(smem_addr(&mbar[i]));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // the previous pass's output is complete and visible after this
  asm volatile("griddepcontrol.wait;" ::: "memory");

  // thread 0: row `row`'s copies into ring slot `slot`, whose previous row was last read before
  // the barrier that ended the previous iteration
  auto issue = [&](int row, int slot) {
    const uint32_t bar = smem_addr(&mbar[slot]);
    const uint32_t dst = smem_addr(ring + slot * ROWB);
    int sy = row;
    bool srow = true, frow = true;
    if (PERIODIC) {
      if (sy < 0) sy += ny;
      if (sy >= ny) sy -= ny;
      if (sy < 0 || sy >= ny) sy = ((row % ny) + ny) % ny;  // chunks taller than the grid
    } else {
      srow = row >= 0 && row < ny;
      frow = row >= -1 && row < ny;
    }
    const uint32_t bytes = (srow ? sbytes : 0u) + (frow ? fbytes : 0u);
    if (bytes == 0) {
      mbar_arrive(bar);
      return;
    }
    mbar_expect_tx(bar, bytes);
    const char* sbase = static_cast<const char*>(p.in) + size_t(sy) * nx * es;
    const float2* fbase = p.faces + size_t((PERIODIC ? sy : row) + 1) * p.pitch_f + 2;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      // (a bounds-checking build skips a copy that leaves its array; the row's wait then runs
      // out and latches its timeout as well)
      if (srow && ss.len[i] > 0 &&
          in_bounds(sy >= 0 && sy < ny && ss.g[i] >= 0 && ss.g[i] + ss.len[i] <= nx, p.status))
        bulk_load(dst + ss.off[i] * es, sbase + size_t(ss.g[i]) * es, ss.len[i] * es, bar);
      if (frow && fs.len[i] > 0 &&
          in_bounds((PERIODIC ? sy : row) + 1 >= 0 && (PERIODIC ? sy : row) + 1 <= ny && fs.g[i] + 2 >= 0 &&
                        fs.g[i] + 2 + fs.len[i] <= p.pitch_f,
                    p.status))
        bulk_load(dst + SB + fs.off[i] * 8, fbase + fs.g[i], fs.len[i] * 8, bar);
    }
  };
  if (tid == 0)
    for (int r = t0; r < min(t0 + L, te + 1); ++r)
      if (!(FAULT && r == t0)) issue(r, r - t0);

  // Dirichlet: which of the thread's columns lie in the grid
  const int gx0 = xs + cx;
  const bool xin0 = PERIODIC || (gx0 >= 0 && gx0 < nx), xin1 = PERIODIC || (gx0 + 1 >= 0 && gx0 + 1 < nx);
  // output columns of this thread: strip columns [h, h + ow) that lie in the grid
  const bool ocol = cx >= p.h && cx < p.h + p.ow && gx0 < nx;
  // the warps whose edge cells this warp's edge lanes read (the strip's outer warps read their
  // own, stale, which only the halo columns see)
  const int wr = w < NW - 1 ? w + 1 : w, wl = w > 0 ? w - 1 : w;

  Cells X[K + 1], Y[K + 1];  // level outputs of alternate iterations (level 0: the loaded row)
  Cells ps[K + 1];           // carried south face flux of each level
  const float2 z2 = make_float2(0.f, 0.f), m1 = make_float2(-1.f, -1.f);
#pragma unroll
  for (int j = 0; j <= K; ++j) {
    X[j].c0 = X[j].c1 = Y[j].c0 = Y[j].c1 = z2;
    ps[j].c0 = ps[j].c1 = z2;
  }
  bool bad = false;
  int timeout = 0;
  int slot = 0;          // ring slot of row t: (t - t0) mod WF_RING
  uint32_t parity = 0;   // parity of that slot's current use

  // a - b exactly, as one packed fused multiply-add
  auto dif = [&](float2 a, float2 b) { return __ffma2_rn(m1, b, a); };

  // One iteration: prev = outputs of iteration t - 1, cur = this iteration's.  Every level runs
  // every iteration: before a level's first needed row (at the chunk start) its rows are unused.
  // Skipping them (a per-level test in every iteration, or a separate code path for the first
  // 2K - 1 iterations) measured slower than the work it saves.
  auto iterate = [&](int t, Cells(&prev)[K + 1], Cells(&cur)[K + 1]) {
    if (tid == 0 && t + L <= te) issue(t + L, (slot + L) & (WF_RING - 1));
    if (!mbar_wait(smem_addr(&mbar[slot]), parity, p.wait_limit)) timeout = 1;
    const unsigned char* rbase = ring + slot * ROWB;
    // level 0: row t of the pass input
    {
      Cells c;
      if (in_real) {
        const float2 u = *reinterpret_cast<const float2*>(rbase + cx * 4);
        c.c0 = make_float2(u.x, 0.f);
        c.c1 = make_float2(u.y, 0.f);
      } else {
        const float4 u = *reinterpret_cast<const float4*>(rbase + cx * 8);
        c.c0 = make_float2(u.x, u.y);
        c.c1 = make_float2(u.z, u.w);
      }
      if (!PERIODIC) {
        const bool yin = t >= 0 && t < ny;
        if (!(yin && xin0)) c.c0 = z2;
        if (!(yin && xin1)) c.c1 = z2;
      }
      cur[0] = c;
    }
    const int par = (t - t0) & 1;
    const float2* eprev = edge + (par ^ 1) * (NW * 2 * KE);
    // warp-uniform loads of the neighbouring warps' edge cells, two levels per 16-byte load
    float2 eRs[KE], eLs[KE];
#pragma unroll
    for (int j = 0; j < KE; j += 2) {
      const float4 a = *reinterpret_cast<const float4*>(eprev + (wr * 2 + 0) * KE + j);
      const float4 b = *reinterpret_cast<const float4*>(eprev + (wl * 2 + 1) * KE + j);
      eRs[j] = make_float2(a.x, a.y);
      eRs[j + 1] = make_float2(a.z, a.w);
      eLs[j] = make_float2(b.x, b.y);
      eLs[j + 1] = make_float2(b.z, b.w);
    }
#pragma unroll
    for (int j = 1; j <= K; ++j) {
      const float2* frow = reinterpret_cast<const float2*>(ring + ((slot - j) & (WF_RING - 1)) * ROWB + SB);
      const float4 F = *reinterpret_cast<const float4*>(frow + cx + 2);  // (ke0, kn0, ke1, kn1)
      const Cells Wp = prev[j - 1], Wn = cur[j - 1];
      const float2 eR = eRs[j - 1], eL = eLs[j - 1];
      const float kw = frow[64 * w + 1].x;  // the warp's west face (warp-uniform)
      // x: east neighbour of the second cell from the next lane (the next warp's edge cell)
      float2 Wr;
      Wr.x = __shfl_down_sync(0xffffffffu, Wp.c0.x, 1);
      Wr.y = __shfl_down_sync(0xffffffffu, Wp.c0.y, 1);
      Wr = lane == 31 ? eR : Wr;
      const float2 de0 = dif(Wp.c1, Wp.c0), de1 = dif(Wr, Wp.c1);
      const float2 Pe0 = scale(F.x, de0), Pe1 = scale(F.z, de1);
      // west flux of the first cell: the previous lane's east flux of its second cell; lane 0
      // forms it from the previous warp's edge cell
      float2 Pw;
      Pw.x = __shfl_up_sync(0xffffffffu, Pe1.x, 1);
      Pw.y = __shfl_up_sync(0xffffffffu, Pe1.y, 1);
      const float2 Pw0 = scale(kw, dif(Wp.c0, eL));
      Pw = lane == 0 ? Pw0 : Pw;
      // y: north difference and flux; the south flux is this level's carry from row t - j - 1
      const float2 Pn0 = scale(F.y, dif(Wn.c0, Wp.c0)), Pn1 = scale(F.w, dif(Wn.c1, Wp.c1));
      const float2 f0 = add2(dif(Pe0, Pw), dif(Pn0, ps[j].c0));
      const float2 f1 = add2(dif(Pe1, Pe0), dif(Pn1, ps[j].c1));
      ps[j].c0 = Pn0;
      ps[j].c1 = Pn1;
      // W += (ca + i cb) f
      const float ca = p.ca[j - 1], cb = p.cb[j - 1];
      const float2 ca2 = make_float2(ca, ca);
      const float2 t0v = __ffma2_rn(ca2, f0, Wp.c0), t1v = __ffma2_rn(ca2, f1, Wp.c1);
      Cells o;
      o.c0 = make_float2(fmaf(-cb, f0.y, t0v.x), fmaf(cb, f0.x, t0v.y));
      o.c1 = make_float2(fmaf(-cb, f1.y, t1v.x), fmaf(cb, f1.x, t1v.y));
      if (!PERIODIC) {
        const int r = t - j;
        const bool yin = r >= 0 && r < ny;
        if (!(yin && xin0)) o.c0 = z2;
        if (!(yin && xin1)) o.c1 = z2;
      }
      cur[j] = o;
    }
    // the pass output: level K's row t - K, rows [y0, y1) of the chunk
    const int r = t - K;
    if (r >= y0 && ocol && in_bounds(size_t(r) * nx + (xs + cx) + 2 <= size_t(nx) * ny, p.status)) {
      const Cells o = cur[K];
      const size_t g = size_t(r) * nx + (xs + cx);
      if (out_real)
        *reinterpret_cast<float2*>(static_cast<float*>(p.out) + g) = make_float2(o.c0.x, o.c1.x);
      else
        *reinterpret_cast<float4*>(static_cast<float2*>(p.out) + g) = make_float4(o.c0.x, o.c0.y, o.c1.x, o.c1.y);
      if (p.check_finite) {
        bad |= (__float_as_uint(o.c0.x) & 0x7f800000u) == 0x7f800000u;
        if (gx0 + 1 < nx) bad |= (__float_as_uint(o.c1.x) & 0x7f800000u) == 0x7f800000u;
      }
    }
    // the warp's edge cells of every level, for the neighbouring warps' next iteration
    float2* enext = edge + par * (NW * 2 * KE);
    if (lane == 0 || lane == 31) {
      float2* e = enext + (w * 2 + (lane == 31)) * KE;
#pragma unroll
      for (int j = 0; j < KE; j += 2) {
        const float2 a = lane == 31 ? cur[j].c1 : cur[j].c0;
        const float2 b = j + 1 < K ? (lane == 31 ? cur[j + 1].c1 : cur[j + 1].c0) : z2;
        *reinterpret_cast<float4*>(e + j) = make_float4(a.x, a.y, b.x, b.y);
      }
    }
    slot = (slot + 1) & (WF_RING - 1);
    parity ^= slot == 0 ? 1u : 0u;
    return __syncthreads_or(timeout);
  };

  int t = t0;
  bool aborted = false;
  while (t <= te) {
    if (iterate(t, X, Y)) {
      aborted = true;
      break;
    }
    ++t;
    if (t > te) break;
    if (iterate(t, Y, X)) {
      aborted = true;
      break;
    }
    ++t;
  }
  if (aborted) {
    // a row never arrived: latch the timeout; wait (bounded) for the copies still in flight
    if (tid == 0) {
      atomicOr(p.status, ST_TIMEOUT);
      for (int r = t; r <= min(te, t + L); ++r) {
        const int rel = r - t0;
        mbar_wait(smem_addr(&mbar[rel & (WF_RING - 1)]), uint32_t((rel / WF_RING) & 1), p.wait_limit);
      }
    }
    return;
  }
  if (bad) atomicOr(p.status, ST_NONFINITE);
}

// (k_east, k_north) of every cell in the padded layout of the wavefront pass, from the face
// arrays fx [ny][nx + 1] and fy [ny + 1][nx]: cell (x, y) at [y + 1][x + 2] for y = -1 .. ny - 1
// and x = -2 .. nx + 1; k_east of column -1 is the west boundary face of column 0, k_north of
// row -1 the south boundary face of row 0; entries outside the faces are zero.
__global__ void k_faces_wf(const float* __restrict__ fx, const float* __restrict__ fy, float2* __restrict__ out,
                           int nx, int ny, int pitch) {
  const size_t total = size_t(ny + 1) * pitch;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < total; i += size_t(gridDim.x) * blockDim.x) {
    const int y = int(i / pitch) - 1, x = int(i % pitch) - 2;
    float2 v = make_float2(0.f, 0.f);
    if (y >= 0 && x >= -1 && x < nx) v.x = fx[size_t(y) * (nx + 1) + (x + 1)];
    if (x >= 0 && x < nx) v.y = fy[size_t(y + 1) * nx + x];
    out[i] = v;
  }
}

size_t smem_bytes(int K) {
  const int CW = 64 * WF_NW;
  const size_t rowb = size_t(CW) * 8 + size_t(CW + 2) * 8;
  const size_t edge = ((2 * WF_NW * 2 * ((K + 1) / 2 * 2) * 8 + 127) / 128) * 128;
  return 256 + edge + size_t(WF_RING) * rowb;
}

// CTAs of one instantiation resident per SM (queried once).
struct WfResidency {
  cudaError_t err;
  int sms, per_sm;
};

template <int K, bool PERIODIC, bool FAULT = false>
cudaError_t launch_k(WfArgs a, cudaStream_t st, bool overlap_previous, int chunk_rows) {
  const auto kern = k_wf2d<K, PERIODIC, FAULT>;
  const size_t smem = smem_bytes(K);
  static const WfResidency res = [kern, smem] {
    WfResidency r{cudaSuccess, 152, 1};
    int dev = 0;
    r.err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (r.err == cudaSuccess) r.err = cudaGetDevice(&dev);
    if (r.err == cudaSuccess) r.err = cudaDeviceGetAttribute(&r.sms, cudaDevAttrMultiProcessorCount, dev);
    if (r.err == cudaSuccess) r.err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r.per_sm, kern, WF_NW * 32, smem);
    if (r.per_sm < 1) r.per_sm = 1;
    return r;
  }();
  if (res.err != cudaSuccess) return res.err;
  const int strips = (a.nx + a.ow - 1) / a.ow;
  if (chunk_rows <= 0) {  // one wave: every resident CTA slot takes one chunk
    const int chunks = std::max(1, std::min(a.ny, (res.sms * res.per_sm) / strips));
    chunk_rows = (a.ny + chunks - 1) / chunks;
  }
  a.H = chunk_rows;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(strips, (a.ny + chunk_rows - 1) / chunk_rows, 1);
  cfg.blockDim = dim3(WF_NW * 32, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = overlap_previous ? 1 : 0;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, a);
  count_launch();
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <int K>
cudaError_t launch_bc(const WfArgs& a, bool periodic, cudaStream_t st, bool ov, int chunk_rows, int fault) {
  if (fault) {  // the fault-injecting instantiation exists for k = 8 only
    if constexpr (K == 8)
      return periodic ? launch_k<K, true, true>(a, st, ov, chunk_rows) : launch_k<K, false, true>(a, st, ov, chunk_rows);
    return cudaErrorInvalidValue;
  }
  return periodic ? launch_k<K, true>(a, st, ov, chunk_rows) : launch_k<K, false>(a, st, ov, chunk_rows);
}

}  // namespace

bool wf2d_k_supported(int k) { return k == 1 || k == 2 || k == 4 || k == 6 || k == 8 || k == 10 || k == 12; }

int wf2d_face_pitch(int nx) { return nx + 4; }

double wf2d_recompute(int nx, int ny, int k) {
  // strips of 256 columns with 2h halo columns; one wave of 3 CTAs per SM (the occupancy of the
  // k <= 8 instantiations); chunks of H rows in which every level runs H + 2k rows
  static const int sms = [] {
    int dev = 0, n = 152;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      n = 152;
    return n;
  }();
  const int h = (k + 3) / 4 * 4, ow = 64 * WF_NW - 2 * h;
  const int strips = (nx + ow - 1) / ow;
  const int chunks = std::max(1, std::min(ny, 3 * sms / strips));
  const int H = (ny + chunks - 1) / chunks;
  return double(strips) * (64 * WF_NW) / nx * double(H + 2 * k) / H;
}

bool wf2d_supported(const frkc2_problem& p, int k, int s, const void* u) {
  const int nx = int(p.n[0]);
  const int last = s % k == 0 ? k : s % k;  // stages of a step's last pass
  return p.ndim == 2 && p.precision == FRKC2_FP32 && p.kappa_kind != FRKC2_KAPPA_POWER && wf2d_k_supported(k) &&
         wf2d_k_supported(last) && nx % 4 == 0 && nx >= 64 * WF_NW && (reinterpret_cast<uintptr_t>(u) & 15) == 0;
}

cudaError_t launch_faces_wf(const frkc2_problem& p, const void* fx, const void* fy, void* out, cudaStream_t st) {
  const int nx = int(p.n[0]), ny = int(p.n[1]), pitch = wf2d_face_pitch(nx);
  const size_t total = size_t(ny + 1) * pitch;
  const int threads = 256;
  const int blocks = int(std::min<size_t>((total + threads - 1) / threads, 152 * 16));
  k_faces_wf<<<blocks, threads, 0, st>>>(static_cast<const float*>(fx), static_cast<const float*>(fy),
                                         static_cast<float2*>(out), nx, ny, pitch);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_pass_wf2d(const frkc2_problem& p, const PassArgs& a, const void* faces_wf, int chunk_rows,
                             bool in_real, bool out_real, cudaStream_t st, bool overlap_previous, long long wait_limit,
                             int fault_inject) {
  (void)p;
  WfArgs w{};
  w.nx = a.nx;
  w.ny = a.ny;
  w.kq = a.k;
  w.h = (a.k + 3) / 4 * 4;
  w.ow = 64 * WF_NW - 2 * w.h;
  w.pitch_f = wf2d_face_pitch(a.nx);
  w.in_real = in_real;
  w.out_real = out_real;
  w.in = a.U_in;
  w.out = a.U_out;
  w.faces = static_cast<const float2*>(faces_wf);
  w.status = a.status;
  w.check_finite = a.check_finite;
  w.wait_limit = wait_limit > 0 ? wait_limit : 1ll << 22;
  for (int j = 0; j < a.k; ++j) {
    w.ca[j] = a.caf[j];
    w.cb[j] = a.cbf[j];
  }
  const bool periodic = a.bc == FRKC2_BC_PERIODIC;
  switch (a.k) {
    case 1: return launch_bc<1>(w, periodic, st, overlap_previous, chunk_rows, fault_inject);
    case 2: return launch_bc<2>(w, periodic, st, overlap_previous, chunk_rows, fault_inject);
    case 4: return launch_bc<4>(w, periodic, st, overlap_previous, chunk_rows, fault_inject);
    case 6: return launch_bc<6>(w, periodic, st, overlap_previous, chunk_rows, fault_inject);
    case 8: return launch_bc<8>(w, periodic, st, overlap_previous, chunk_rows, fault_inject);
    case 10: return launch_bc<10>(w, periodic, st, overlap_previous, chunk_rows, fault_inject);
    case 12: return launch_bc<12>(w, periodic, st, overlap_previous, chunk_rows, fault_inject);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace frkc2
