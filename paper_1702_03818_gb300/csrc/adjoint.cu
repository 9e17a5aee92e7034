// Discrete adjoint of the FRKC2 step (reverse replay of the stages of Sec. 3, Eq. 13).
//
// Forward stage: W^{l+1} = W^l + c_l f(W^l), c_l = dt a_l.  With the real inner product
// <x, y> = Re(x^H y) its adjoint is lam^l = lam^{l+1} + conj(c_l) J_f(W^l)^H lam^{l+1}, where
// for the flux-form operator
//   (J^H lam)_m = (1/dx^2) sum_{nb i of m} (lam_i - lam_m) conj(kappa_f - kappa'(W_m)(W_i - W_m)/2)
// (kappa' = 0 for a fixed conductivity, which makes J^H the operator itself).  For a
// conductivity field the stage also contributes to dJ/dkappa: the face between m and i
// receives Re(c_l conj(lam_m - lam_i)(W_i - W_m)) / dx^2, and passes half of it to each cell
// (a Dirichlet boundary face, whose conductivity is its interior cell's, passes all of it).
//
// Driver: the forward run keeps the state every ckpt_every steps; each segment of steps is
// recomputed from its checkpoint with every stage state written to a tape in the workspace,
// then the segment's stages are reversed (last step first, last stage first).  The last
// segment's tape is still in place after the forward run and is not recomputed.  2D problems
// with a fixed conductivity use the streaming kernels with the tape and lambda stored
// interleaved (U, V) -- in FP32 the temporally blocked tape and reverse passes of
// adjoint_tb2d.cu, 8 stages each; the others use the tile kernels with planar U, V.
#include <algorithm>
#include <cmath>

#include <cuda_runtime.h>

#include "frkc2.h"
#include "frkc2_internal.h"
#include "frkc2_math.cuh"

namespace frkc2 {

frkc2_status validate_problem(const frkc2_problem* p);

namespace {

constexpr int ADJ_THREADS = 256;

struct AdjArgs {
  int ndim, bc;
  int nx, ny, nz;
  int tx, ty, tz;
  const void* WU;      // stage state W^l
  const void* WV;      // nullptr = zero imaginary part (stage 0)
  const void* LU_in;   // lam^{l+1}
  const void* LV_in;   // nullptr = zero
  void* LU_out;        // lam^l
  void* LV_out;
  const void* fx;
  const void* fy;
  const void* fz;
  double* dk;          // dJ/dkappa accumulator (FIELD) or nullptr
  double kc, kp;
  double ca, cb;       // c_l / dx^2 = dt (alpha_l + i beta_l) / dx^2
};

__device__ __forceinline__ int wrap_i(int g, int n) {
  int r = g % n;
  return r < 0 ? r + n : r;
}

// kappa'(w) = c p w^(p-1) on the principal branch (0 at w = 0).
template <class T>
__device__ __forceinline__ void dkappa_power(T u, T v, T c, T p, T& dr, T& di) {
  dr = T(0);
  di = T(0);
  if (u == T(0) && v == T(0)) return;
  T wr, wi;
  if (p == T(2.5)) {  // w^1.5 = w sqrt(w)
    T sr, si;
    csqrt_principal<T>(u, v, sr, si);
    wr = u * sr - v * si;
    wi = u * si + v * sr;
  } else {
    const T r = hypot(u, v), th = atan2(v, u);
    const T rp = pow(r, p - T(1));
    T sn, cs;
    sincos((p - T(1)) * th, &sn, &cs);
    wr = rp * cs;
    wi = rp * sn;
  }
  dr = c * p * wr;
  di = c * p * wi;
}

template <class S, class A, bool POWER>
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_generic(const AdjArgs p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int hx = 1, hy = p.ndim >= 2 ? 1 : 0, hz = p.ndim >= 3 ? 1 : 0;
  const int RX = p.tx + 2 * hx, RY = p.ty + 2 * hy, RZ = p.tz + 2 * hz;
  const int plane = RX * RY, R = plane * RZ;
  S* wu = reinterpret_cast<S*>(smem);
  S* wv = wu + R;
  S* lu = wv + R;
  S* lv = lu + R;
  A* f0 = reinterpret_cast<A*>(lv + R);  // x faces, or Re kappa(W)
  A* f1 = f0 + R;                        // y faces, or Im kappa(W)
  A* f2 = f1 + R;                        // z faces
  const bool periodic = p.bc == FRKC2_BC_PERIODIC;
  const int x0 = blockIdx.x * p.tx - hx, y0 = blockIdx.y * p.ty - hy, z0 = blockIdx.z * p.tz - hz;
  const S* __restrict__ WU = static_cast<const S*>(p.WU);
  const S* __restrict__ WV = static_cast<const S*>(p.WV);
  const S* __restrict__ LU = static_cast<const S*>(p.LU_in);
  const S* __restrict__ LV = static_cast<const S*>(p.LV_in);
  const A* __restrict__ FX = static_cast<const A*>(p.fx);
  const A* __restrict__ FY = static_cast<const A*>(p.fy);
  const A* __restrict__ FZ = static_cast<const A*>(p.fz);
  const int tid = threadIdx.x;

  for (int idx = tid; idx < R; idx += ADJ_THREADS) {
    const int z = idx / plane, rem = idx - z * plane, y = rem / RX, x = rem - y * RX;
    const int gx = x0 + x, gy = y0 + y, gz = z0 + z;
    S a = S(0), b = S(0), c = S(0), d = S(0);
    A q0 = A(0), q1 = A(0), q2 = A(0);
    bool inside;
    int wx, wy, wz;
    if (periodic) {
      wx = wrap_i(gx, p.nx);
      wy = wrap_i(gy, p.ny);
      wz = wrap_i(gz, p.nz);
      inside = true;
    } else {
      wx = gx;
      wy = gy;
      wz = gz;
      inside = gx >= 0 && gx < p.nx && gy >= 0 && gy < p.ny && gz >= 0 && gz < p.nz;
    }
    if (inside) {
      const size_t g = (size_t(wz) * p.ny + wy) * p.nx + wx;
      a = WU[g];
      if (WV) b = WV[g];
      c = LU[g];
      if (LV) d = LV[g];
    }
    if (!POWER) {
      if (periodic) {
        q0 = FX[(size_t(wz) * p.ny + wy) * (p.nx + 1) + wx];
        if (p.ndim >= 2) q1 = FY[(size_t(wz) * (p.ny + 1) + wy) * p.nx + wx];
        if (p.ndim >= 3) q2 = FZ[(size_t(wz) * p.ny + wy) * p.nx + wx];
      } else {
        const bool inx = gx >= 0 && gx < p.nx, iny = gy >= 0 && gy < p.ny, inz = gz >= 0 && gz < p.nz;
        if (iny && inz && gx >= 0 && gx <= p.nx) q0 = FX[(size_t(gz) * p.ny + gy) * (p.nx + 1) + gx];
        if (p.ndim >= 2 && inx && inz && gy >= 0 && gy <= p.ny) q1 = FY[(size_t(gz) * (p.ny + 1) + gy) * p.nx + gx];
        if (p.ndim >= 3 && inx && iny && gz >= 0 && gz <= p.nz) q2 = FZ[(size_t(gz) * p.ny + gy) * p.nx + gx];
      }
    } else {
      kappa_power<A>(A(a), A(b), A(p.kc), A(p.kp), q0, q1);  // ghost: w = 0 -> kappa = 1
    }
    wu[idx] = a;
    wv[idx] = b;
    lu[idx] = c;
    lv[idx] = d;
    f0[idx] = q0;
    if (POWER || p.ndim >= 2) f1[idx] = q1;
    if (!POWER && p.ndim >= 3) f2[idx] = q2;
  }
  __syncthreads();

  S* __restrict__ LUo = static_cast<S*>(p.LU_out);
  S* __restrict__ LVo = static_cast<S*>(p.LV_out);
  const int ox = blockIdx.x * p.tx, oy = blockIdx.y * p.ty, oz = blockIdx.z * p.tz;
  const int ex = min(p.tx, p.nx - ox), ey = min(p.ty, p.ny - oy), ez = min(p.tz, p.nz - oz);
  const int st[3] = {1, RX, plane};
  for (int t = tid; t < ex * ey * ez; t += ADJ_THREADS) {
    const int z = t / (ex * ey), r = t - z * ex * ey, y = r / ex, x = r - y * ex;
    const int m = (z + hz) * plane + (y + hy) * RX + (x + hx);
    const int gx = ox + x, gy = oy + y, gz = oz + z;
    const S Wm_r = wu[m], Wm_i = wv[m], Lm_r = lu[m], Lm_i = lv[m];
    A dkr = A(0), dki = A(0);
    if (POWER) dkappa_power<A>(A(Wm_r), A(Wm_i), A(p.kc), A(p.kp), dkr, dki);
    A ar = A(0), ai = A(0);
    double g = 0.0;
    const int gc[3] = {gx, gy, gz};
    const int nn[3] = {p.nx, p.ny, p.nz};
#pragma unroll
    for (int dd = 0; dd < 3; ++dd) {
      if (dd >= p.ndim) break;
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const int i = side ? m + st[dd] : m - st[dd];
        const A dlr = A(lu[i] - Lm_r), dli = A(lv[i] - Lm_i);
        const A dWr = A(wu[i] - Wm_r), dWi = A(wv[i] - Wm_i);
        if (!POWER) {
          const A* F = dd == 0 ? f0 : (dd == 1 ? f1 : f2);
          const A kf = side ? F[i] : F[m];
          ar += kf * dlr;
          ai += kf * dli;
          if (p.dk) {
            const double zr = double(dlr) * double(dWr) + double(dli) * double(dWi);
            const double zi = double(dlr) * double(dWi) - double(dli) * double(dWr);
            const double G = -(p.ca * zr - p.cb * zi);
            const int gn = side ? gc[dd] + 1 : gc[dd] - 1;
            const bool ghost = !periodic && (gn < 0 || gn >= nn[dd]);
            g += (ghost ? 1.0 : 0.5) * G;
          }
        } else {
          // t = kappa_f - kappa'(W_m) (W_i - W_m) / 2
          const A tr = A(0.5) * (f0[m] + f0[i]) - A(0.5) * (dkr * dWr - dki * dWi);
          const A ti = A(0.5) * (f1[m] + f1[i]) - A(0.5) * (dkr * dWi + dki * dWr);
          ar += dlr * tr + dli * ti;
          ai += dli * tr - dlr * ti;
        }
      }
    }
    const size_t gidx = (size_t(gz) * p.ny + gy) * p.nx + gx;
    const S ca = S(p.ca), cb = S(p.cb);
    LUo[gidx] = Lm_r + ca * S(ar) + cb * S(ai);
    LVo[gidx] = Lm_i + ca * S(ai) - cb * S(ar);
    if (p.dk) p.dk[gidx] += g;
  }
}

size_t adj_smem_bytes(const frkc2_problem& pr, int tx, int ty, int tz) {
  const size_t R = size_t(tx + 2) * (pr.ndim >= 2 ? ty + 2 : 1) * (pr.ndim >= 3 ? tz + 2 : 1);
  const size_t S = state_bytes(pr.precision), A = arith_bytes(pr.precision);
  const size_t nf = pr.kappa_kind == FRKC2_KAPPA_POWER ? 2 : size_t(pr.ndim);
  return R * (4 * S + nf * A);
}

template <class S, class A, bool POWER>
cudaError_t launch_adj_t(const AdjArgs& a, size_t smem, cudaStream_t st) {
  auto kern = k_adj_generic<S, A, POWER>;
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
  }
  dim3 grid((a.nx + a.tx - 1) / a.tx, (a.ny + a.ty - 1) / a.ty, (a.nz + a.tz - 1) / a.tz);
  kern<<<grid, ADJ_THREADS, smem, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_adj(const frkc2_problem& pr, const AdjArgs& a, cudaStream_t st) {
  const size_t smem = adj_smem_bytes(pr, a.tx, a.ty, a.tz);
  const bool power = pr.kappa_kind == FRKC2_KAPPA_POWER;
  switch (pr.precision) {
    case FRKC2_FP64:
      return power ? launch_adj_t<double, double, true>(a, smem, st) : launch_adj_t<double, double, false>(a, smem, st);
    case FRKC2_FP32:
      return power ? launch_adj_t<float, float, true>(a, smem, st) : launch_adj_t<float, float, false>(a, smem, st);
    default:
      return power ? launch_adj_t<double, float, true>(a, smem, st) : launch_adj_t<double, float, false>(a, smem, st);
  }
}

template <class A>
__global__ void k_store_grad(const double* __restrict__ acc, A* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    out[i] = A(acc[i]);
}

struct AdjLayout {
  size_t status, fx, fy, fz, fen, ckpt, tape, lam, dk, total;
  int nseg;
};

AdjLayout adj_layout(const frkc2_problem& p, int s, int nsteps, int c) {
  AdjLayout L{};
  const FaceLayout F = faces_layout(p);
  const size_t A = arith_bytes(p.precision), S = state_bytes(p.precision), N = cells(p);
  L.nseg = (nsteps + c - 1) / c;
  size_t off = 256;
  L.status = 0;
  L.fx = off;
  off += align256(F.nfx * A);
  L.fy = off;
  off += align256(F.nfy * A);
  L.fz = off;
  off += align256(F.nfz * A);
  L.fen = off;
  if (p.ndim == 2 && p.kappa_kind != FRKC2_KAPPA_POWER) off += align256(face_pair_bytes(p));
  L.ckpt = off;  // nseg + 1 real states
  off += size_t(L.nseg + 1) * align256(N * S);
  L.tape = off;  // c steps x s stages x (U, V)
  off += size_t(c) * s * 2 * align256(N * S);
  L.lam = off;   // two complex adjoint buffers
  off += 4 * align256(N * S);
  L.dk = off;
  off += align256(N * sizeof(double));
  L.total = off;
  return L;
}


// Shared state of one adjoint computation (forward with checkpoints, then backward).
struct AdjCtx {
  const frkc2_plan_s* plan;
  const frkc2_problem* p;
  double dt, h2;
  int nsteps, c, s;
  AdjLayout L;
  char* base;
  cudaStream_t st;
  size_t N, SB, slot;
  bool stream2d;  // 2D fixed conductivity: streaming kernels, interleaved tape and lambda
  bool tb;        // ... in FP32: temporally blocked tape and reverse passes of tbk stages
  int tbk;
  int tx, ty, tz;
  char* ckpt(int j) const { return base + L.ckpt + size_t(j) * slot; }
  char* tape(int q, int l) const { return base + L.tape + (size_t(q) * s + l) * 2 * slot; }
  // W^0 of step q of segment j: the checkpoint for the first step, else tape slot 0
  char* w0(int j, int q) const { return q == 0 ? ckpt(j) : tape(q, 0); }
};

frkc2_status adj_setup(AdjCtx& C, frkc2_plan_t plan, const frkc2_problem* prob, double dt, int nsteps,
                       int ckpt_every, void* ws, size_t ws_bytes, void* stream) {
  if (!plan || !ws || nsteps < 1 || ckpt_every < 1) return FRKC2_EINVAL;
  const frkc2_status v = validate_problem(prob);
  if (v != FRKC2_OK) return v;
  if (prob->precision == FRKC2_DFLOAT) return FRKC2_EUNSUPPORTED;
  if (!(dt > 0.0) || !std::isfinite(dt)) return FRKC2_EINVAL;
  if (reinterpret_cast<uintptr_t>(ws) & 255) return FRKC2_EINVAL;
  const frkc2_problem& p = *prob;
  C.plan = plan;
  C.p = prob;
  C.dt = dt;
  C.h2 = p.dx * p.dx;
  C.nsteps = nsteps;
  C.s = plan->s;
  C.c = std::min(ckpt_every, nsteps);
  C.L = adj_layout(p, C.s, nsteps, C.c);
  if (ws_bytes < C.L.total) return FRKC2_ENOMEM;
  C.base = static_cast<char*>(ws);
  C.st = static_cast<cudaStream_t>(stream);
  C.N = cells(p);
  C.SB = state_bytes(p.precision);
  C.slot = align256(C.N * C.SB);
  C.stream2d = p.ndim == 2 && p.kappa_kind != FRKC2_KAPPA_POWER;
  C.tbk = 8;
  C.tb = C.stream2d && adj_tb2d_supported(p, C.tbk);
  default_tiles(p, 1, &C.tx, &C.ty, &C.tz);
  if (p.ndim < 2) C.ty = 1;
  if (p.ndim < 3) C.tz = 1;
  if (!C.stream2d && adj_smem_bytes(p, C.tx, C.ty, C.tz) > 200 * 1024) return FRKC2_EINVAL;
  return FRKC2_OK;
}

// Recompute segment j from its checkpoint, every stage state to the tape; the segment's final
// state goes to checkpoint j + 1.
bool run_segment(const AdjCtx& C, int j) {
  const frkc2_problem& p = *C.p;
  PassArgs a{};
  a.ndim = p.ndim;
  a.bc = p.bc;
  a.nx = int(p.n[0]);
  a.ny = int(p.n[1]);
  a.nz = int(p.n[2]);
  a.tx = C.tx;
  a.ty = C.ty;
  a.tz = C.tz;
  a.k = 1;
  a.hx = 1;
  a.hy = p.ndim >= 2 ? 1 : 0;
  a.hz = p.ndim >= 3 ? 1 : 0;
  a.fx = C.base + C.L.fx;
  a.fy = C.base + C.L.fy;
  a.fz = C.base + C.L.fz;
  a.kc = p.kappa_c;
  a.kp = p.kappa_p;
  a.status = reinterpret_cast<unsigned*>(C.base + C.L.status);
  const int n0 = j * C.c, m = std::min(C.c, C.nsteps - n0);
  if (C.tb) {
    for (int q = 0; q < m; ++q)
      for (int l0 = 0; l0 < C.s;) {
        AdjTbPass t{};
        t.nst = std::min(C.tbk, C.s - l0);
        t.in = l0 == 0 ? C.w0(j, q) : C.tape(q, l0);
        t.in_complex = l0 != 0;
        for (int jj = 0; jj < t.nst; ++jj) {
          const int l = l0 + jj;
          t.out[jj] = l + 1 < C.s ? C.tape(q, l + 1) : (q + 1 < m ? C.tape(q + 1, 0) : C.ckpt(j + 1));
          t.ca[jj] = C.dt * C.plan->a_re[l] / C.h2;
          t.cb[jj] = C.dt * C.plan->a_im[l] / C.h2;
        }
        t.last_real = l0 + t.nst == C.s;
        if (launch_tape_tb2d(p, C.tbk, t, C.base + C.L.fx, C.base + C.L.fy, a.status, C.st) != cudaSuccess)
          return false;
        l0 += t.nst;
      }
    return true;
  }
  for (int q = 0; q < m; ++q) {
    for (int l = 0; l < C.s; ++l) {
      const bool last = l + 1 == C.s;
      char* in = l == 0 ? C.w0(j, q) : C.tape(q, l);
      char* out = !last ? C.tape(q, l + 1) : (q + 1 < m ? C.tape(q + 1, 0) : C.ckpt(j + 1));
      a.U_in = in;
      a.U_out = out;
      a.check_finite = last;
      a.ca[0] = C.dt * C.plan->a_re[l] / C.h2;
      a.cb[0] = C.dt * C.plan->a_im[l] / C.h2;
      cudaError_t e;
      if (C.stream2d) {
        a.V_in = nullptr;
        a.V_out = nullptr;
        a.in_mode = l == 0 ? PASS_IO_REAL : PASS_IO_COMPLEX;
        a.out_mode = last ? PASS_IO_REAL : PASS_IO_COMPLEX;
        e = launch_pass_stream2d(p, a, C.base + C.L.fen, C.st);
      } else {
        a.V_in = l == 0 ? nullptr : in + C.slot;
        a.V_out = last ? nullptr : out + C.slot;
        e = launch_pass_generic(p, a, C.st);
      }
      if (e != cudaSuccess) return false;
    }
  }
  return true;
}

// Segment j without a tape (FP32 register-tiled path): the forward passes of frkc2_step from
// checkpoint j to checkpoint j + 1, planar (U, V) ping-pong buffers in the tape area (the
// segments before the last leave no tape the backward reads: it recomputes each from its
// checkpoint).
bool run_segment_plain_tb(const AdjCtx& C, int j) {
  const frkc2_problem& p = *C.p;
  PassArgs a{};
  a.ndim = 2;
  a.bc = p.bc;
  a.nx = int(p.n[0]);
  a.ny = int(p.n[1]);
  a.nz = 1;
  a.fx = C.base + C.L.fx;
  a.fy = C.base + C.L.fy;
  a.kc = p.kappa_c;
  a.kp = p.kappa_p;
  a.status = reinterpret_cast<unsigned*>(C.base + C.L.status);
  char* ua = C.tape(0, 0);
  char* va = ua + C.slot;
  char* ub = C.tape(0, 1);
  char* vb = ub + C.slot;
  const void* curU = C.ckpt(j);
  const void* curV = nullptr;
  const int n0 = j * C.c, m = std::min(C.c, C.nsteps - n0);
  const int k = C.tbk, npass = (C.s + k - 1) / k;
  for (int q = 0; q < m; ++q)
    for (int ps = 0; ps < npass; ++ps) {
      const int l0 = ps * k, kq = std::min(k, C.s - l0);
      const bool last = ps == npass - 1;
      void* outU = (last && q == m - 1) ? static_cast<void*>(C.ckpt(j + 1)) : (curU == ua ? ub : ua);
      void* outV = last ? nullptr : (curV == va ? vb : va);
      a.k = kq;
      a.hx = kq;
      a.hy = kq;
      a.U_in = curU;
      a.V_in = curV;
      a.U_out = outU;
      a.V_out = outV;
      a.check_finite = last ? 1 : 0;
      for (int jj = 0; jj < kq; ++jj) {
        a.ca[jj] = C.dt * C.plan->a_re[l0 + jj] / C.h2;
        a.cb[jj] = C.dt * C.plan->a_im[l0 + jj] / C.h2;
        a.caf[jj] = float(a.ca[jj]);
        a.cbf[jj] = float(a.cb[jj]);
      }
      a.in_mode = curV ? PASS_IO_PLANAR : PASS_IO_REAL;
      a.out_mode = outV ? PASS_IO_PLANAR : PASS_IO_REAL;
      if (launch_pass_tb2d(p, a, C.st, q > 0 || ps > 0) != cudaSuccess) return false;
      curU = outU;
      curV = outV;
    }
  return true;
}

frkc2_status adj_forward(const AdjCtx& C, const void* u0) {
  const frkc2_problem& p = *C.p;
  if (p.kappa_kind != FRKC2_KAPPA_POWER) {
    if (launch_faces(p, C.base + C.L.fx, C.base + C.L.fy, C.base + C.L.fz, C.st) != cudaSuccess) return FRKC2_ECUDA;
    if (p.ndim == 2 && launch_face_pairs(p, C.base + C.L.fx, C.base + C.L.fy, C.base + C.L.fen, C.st) != cudaSuccess)
      return FRKC2_ECUDA;
  }
  if (cudaMemcpyAsync(C.ckpt(0), u0, C.N * C.SB, cudaMemcpyDeviceToDevice, C.st) != cudaSuccess) return FRKC2_ECUDA;
  // the last segment's tape stays for the backward; in FP32 the segments before it run the
  // forward passes alone (the tape passes write 8 bytes per cell-stage more)
  for (int j = 0; j < C.L.nseg; ++j)
    if (!(C.tb && j + 1 < C.L.nseg && C.s >= 2 ? run_segment_plain_tb(C, j) : run_segment(C, j))) return FRKC2_ECUDA;
  return FRKC2_OK;
}

frkc2_status adj_backward(const AdjCtx& C, const void* g, void* dJdu0, void* dJdkappa) {
  const frkc2_problem& p = *C.p;
  double* dk = dJdkappa ? reinterpret_cast<double*>(C.base + C.L.dk) : nullptr;
  if (dk && cudaMemsetAsync(dk, 0, C.N * sizeof(double), C.st) != cudaSuccess) return FRKC2_ECUDA;
  char* lam[2] = {C.base + C.L.lam, C.base + C.L.lam + 2 * C.slot};  // each: U then V (planar) or (U,V) pairs
  int cur = 0;
  bool lam_real_input = true;  // g itself for the last step
  const void* lam_src = g;
  AdjArgs b{};
  b.ndim = p.ndim;
  b.bc = p.bc;
  b.nx = int(p.n[0]);
  b.ny = int(p.n[1]);
  b.nz = int(p.n[2]);
  b.tx = C.tx;
  b.ty = C.ty;
  b.tz = C.tz;
  b.fx = C.base + C.L.fx;
  b.fy = C.base + C.L.fy;
  b.fz = C.base + C.L.fz;
  b.dk = dk;
  b.kc = p.kappa_c;
  b.kp = p.kappa_p;
  AdjStreamArgs sa{};
  sa.nx = int(p.n[0]);
  sa.ny = int(p.n[1]);
  sa.fen = C.base + C.L.fen;
  sa.dk = dk;
  for (int j = C.L.nseg - 1; j >= 0; --j) {
    if (j != C.L.nseg - 1 && !run_segment(C, j)) return FRKC2_ECUDA;
    const int m = std::min(C.c, C.nsteps - j * C.c);
    for (int q = m - 1; q >= 0; --q) {
      if (C.tb) {  // passes of up to tbk stages, last stage first
        for (int lhi = C.s; lhi > 0;) {
          AdjTbPass t{};
          t.nst = std::min(C.tbk, lhi);
          for (int jj = 0; jj < t.nst; ++jj) {
            const int l = lhi - 1 - jj;
            t.W[jj] = l == 0 ? C.w0(j, q) : C.tape(q, l);
            t.w_complex[jj] = l != 0;
            t.ca[jj] = C.dt * C.plan->a_re[l] / C.h2;
            t.cb[jj] = C.dt * C.plan->a_im[l] / C.h2;
          }
          if (lhi == C.s) {  // the step output is Re W^L: a real lambda
            t.L_in = lam_src;
            t.l_mode = lam_real_input ? 0 : 2;
          } else {
            t.L_in = lam[cur];
            t.l_mode = 1;
          }
          t.L_out = lam[cur ^ 1];
          t.dk = dk;
          if (launch_adjrev_tb2d(p, C.tbk, t, C.base + C.L.fx, C.base + C.L.fy,
                                 reinterpret_cast<unsigned*>(C.base + C.L.status), C.st) != cudaSuccess)
            return FRKC2_ECUDA;
          cur ^= 1;
          lhi -= t.nst;
        }
        lam_src = lam[cur];
        lam_real_input = false;
        continue;
      }
      // the step output is Re W^L: the adjoint of a step starts from a real lambda
      for (int l = C.s - 1; l >= 0; --l) {
        const bool first = l == C.s - 1;
        char* W = l == 0 ? C.w0(j, q) : C.tape(q, l);
        const double ca = C.dt * C.plan->a_re[l] / C.h2, cb = C.dt * C.plan->a_im[l] / C.h2;
        cudaError_t e;
        if (C.stream2d) {
          sa.W = W;
          sa.w_complex = l == 0 ? 0 : 1;
          if (first) {
            sa.L_in = lam_src;
            sa.l_complex = lam_real_input ? 0 : 2;  // 2: real part of an interleaved buffer
          } else {
            sa.L_in = lam[cur];
            sa.l_complex = 1;
          }
          sa.L_out = lam[cur ^ 1];
          sa.ca = ca;
          sa.cb = cb;
          e = launch_adj_stream2d(p, sa, C.st);
        } else {
          b.WU = W;
          b.WV = l == 0 ? nullptr : W + C.slot;
          if (first) {
            b.LU_in = lam_src;
            b.LV_in = nullptr;
          } else {
            b.LU_in = lam[cur];
            b.LV_in = lam[cur] + C.slot;
          }
          b.LU_out = lam[cur ^ 1];
          b.LV_out = lam[cur ^ 1] + C.slot;
          b.ca = ca;
          b.cb = cb;
          e = launch_adj(p, b, C.st);
        }
        if (e != cudaSuccess) return FRKC2_ECUDA;
        cur ^= 1;
      }
      lam_src = lam[cur];
      lam_real_input = false;
    }
  }
  // dJ/du0 = Re lam^0
  if (C.stream2d) {
    if (cudaMemcpy2DAsync(dJdu0, C.SB, lam[cur], 2 * C.SB, C.SB, C.N, cudaMemcpyDeviceToDevice, C.st) != cudaSuccess)
      return FRKC2_ECUDA;
  } else {
    if (cudaMemcpyAsync(dJdu0, lam[cur], C.N * C.SB, cudaMemcpyDeviceToDevice, C.st) != cudaSuccess)
      return FRKC2_ECUDA;
  }
  if (dJdkappa) {
    const int threads = 256, blocks = int(std::min<size_t>((C.N + threads - 1) / threads, 4096));
    if (p.precision == FRKC2_FP64)
      k_store_grad<double><<<blocks, threads, 0, C.st>>>(dk, static_cast<double*>(dJdkappa), C.N);
    else
      k_store_grad<float><<<blocks, threads, 0, C.st>>>(dk, static_cast<float*>(dJdkappa), C.N);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return FRKC2_ECUDA;
  }
  return FRKC2_OK;
}

}  // namespace
}  // namespace frkc2

using namespace frkc2;

extern "C" {

frkc2_status frkc2_adjoint_workspace_size(const frkc2_plan_t plan, const frkc2_problem* prob, int nsteps,
                                          int ckpt_every, size_t* bytes) {
  if (!plan || !bytes || nsteps < 0 || ckpt_every < 1) return FRKC2_EINVAL;
  const frkc2_status v = validate_problem(prob);
  if (v != FRKC2_OK) return v;
  if (prob->precision == FRKC2_DFLOAT) return FRKC2_EUNSUPPORTED;
  const int n = std::max(nsteps, 1);
  *bytes = adj_layout(*prob, plan->s, n, std::min(ckpt_every, n)).total;
  return FRKC2_OK;
}

frkc2_status frkc2_adjoint_forward(frkc2_plan_t plan, const frkc2_problem* prob, double dt, int nsteps,
                                   int ckpt_every, const void* u0, void* uT, void* ws, size_t ws_bytes,
                                   void* stream) {
  const frkc2::NvtxRange call_range("frkc2_adjoint_forward");
  if (!u0) return FRKC2_EINVAL;
  AdjCtx C;
  frkc2_status v = adj_setup(C, plan, prob, dt, nsteps, ckpt_every, ws, ws_bytes, stream);
  if (v != FRKC2_OK) return v;
  v = adj_forward(C, u0);
  if (v != FRKC2_OK) return v;
  if (uT && cudaMemcpyAsync(uT, C.ckpt(C.L.nseg), C.N * C.SB, cudaMemcpyDeviceToDevice, C.st) != cudaSuccess)
    return FRKC2_ECUDA;
  return FRKC2_OK;
}

frkc2_status frkc2_adjoint_backward(frkc2_plan_t plan, const frkc2_problem* prob, double dt, int nsteps,
                                    int ckpt_every, const void* g, void* dJdu0, void* dJdkappa, void* ws,
                                    size_t ws_bytes, void* stream) {
  const frkc2::NvtxRange call_range("frkc2_adjoint_backward");
  if (!g || !dJdu0) return FRKC2_EINVAL;
  if (dJdkappa && (!prob || prob->kappa_kind != FRKC2_KAPPA_FIELD)) return FRKC2_EINVAL;
  AdjCtx C;
  const frkc2_status v = adj_setup(C, plan, prob, dt, nsteps, ckpt_every, ws, ws_bytes, stream);
  if (v != FRKC2_OK) return v;
  return adj_backward(C, g, dJdu0, dJdkappa);
}

frkc2_status frkc2_adjoint(frkc2_plan_t plan, const frkc2_problem* prob, double dt, int nsteps, int ckpt_every,
                           const void* u0, const void* g, void* dJdu0, void* dJdkappa, void* ws, size_t ws_bytes,
                           void* stream) {
  const frkc2::NvtxRange call_range("frkc2_adjoint");
  if (!u0 || !g || !dJdu0) return FRKC2_EINVAL;
  if (dJdkappa && (!prob || prob->kappa_kind != FRKC2_KAPPA_FIELD)) return FRKC2_EINVAL;
  AdjCtx C;
  frkc2_status v = adj_setup(C, plan, prob, dt, nsteps, ckpt_every, ws, ws_bytes, stream);
  if (v != FRKC2_OK) return v;
  v = adj_forward(C, u0);
  if (v != FRKC2_OK) return v;
  return adj_backward(C, g, dJdu0, dJdkappa);
}

}  // extern "C"
