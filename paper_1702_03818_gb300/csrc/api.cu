// C ABI entry points for the forward step, the spectral-radius bound and the workspace.
#include <algorithm>
#include <cmath>
#include <cstring>

#include <cuda_runtime.h>

#include "frkc2.h"
#include "frkc2_internal.h"

namespace frkc2 {

static thread_local long long g_launches = 0;

void count_launch(int n) { g_launches += n; }

size_t state_bytes(int precision) { return precision == FRKC2_FP32 ? 4 : 8; }
size_t arith_bytes(int precision) { return precision == FRKC2_FP64 ? 8 : 4; }
size_t cells(const frkc2_problem& p) { return size_t(p.n[0]) * size_t(p.n[1]) * size_t(p.n[2]); }

FaceLayout faces_layout(const frkc2_problem& p) {
  FaceLayout L{0, 0, 0};
  if (p.kappa_kind == FRKC2_KAPPA_POWER) return L;
  const size_t nx = p.n[0], ny = p.n[1], nz = p.n[2];
  L.nfx = nz * ny * (nx + 1);
  if (p.ndim >= 2) L.nfy = nz * (ny + 1) * nx;
  if (p.ndim >= 3) L.nfz = (nz + 1) * ny * nx;
  return L;
}

StepLayout step_layout(const frkc2_problem& p) {
  StepLayout s{};
  const FaceLayout F = faces_layout(p);
  const size_t A = arith_bytes(p.precision), S = state_bytes(p.precision), N = cells(p);
  size_t off = 0;
  s.status = off;
  off += 256;
  s.fx = off;
  off += align256(F.nfx * A);
  s.fy = off;
  off += align256(F.nfy * A);
  s.fz = off;
  off += align256(F.nfz * A);
  s.fen = off;  // face pairs of the 2D streaming pass
  if (p.ndim == 2 && p.kappa_kind != FRKC2_KAPPA_POWER) off += align256(face_pair_bytes(p));
  s.ua = off;
  off += align256(N * S);
  s.va = off;
  off += align256(N * S);
  s.ub = off;
  off += align256(N * S);
  s.vb = off;
  off += align256(N * S);
  s.total = off;
  return s;
}

void default_tiles(const frkc2_problem& p, int k, int* tx, int* ty, int* tz) {
  if (p.ndim == 1) {
    *tx = 1024;
    *ty = *tz = 1;
  } else if (p.ndim == 2) {
    *tx = 64;
    *ty = p.precision == FRKC2_FP32 ? 32 : 16;
    *tz = 1;
  } else {
    *tx = 32;
    *ty = 4;
    *tz = k > 1 ? 2 : 4;
  }
}

static int default_k(const frkc2_problem& p) {
  if (p.ndim == 1) return 16;
  if (p.ndim == 2 && p.kappa_kind != FRKC2_KAPPA_POWER) {
    if (p.precision == FRKC2_FP32) return 8;
    if (p.precision == FRKC2_DFLOAT) return 8;
  }
  return 1;
}

static int smem_optin() {
  static const int v = [] {
    int dev = 0, r = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&r, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      r = 227 * 1024;
    return r;
  }();
  return v;
}

frkc2_status validate_problem(const frkc2_problem* p) {
  if (!p) return FRKC2_EINVAL;
  if (p->ndim < 1 || p->ndim > 3) return FRKC2_EINVAL;
  if (p->bc != FRKC2_BC_PERIODIC && p->bc != FRKC2_BC_DIRICHLET) return FRKC2_EINVAL;
  if (p->kappa_kind < FRKC2_KAPPA_CONST || p->kappa_kind > FRKC2_KAPPA_POWER) return FRKC2_EINVAL;
  if (p->precision < FRKC2_FP64 || p->precision > FRKC2_DFLOAT) return FRKC2_EINVAL;
  for (int d = 0; d < 3; ++d) {
    if (p->n[d] < 1 || p->n[d] > (int64_t(1) << 30)) return FRKC2_EINVAL;
    if (d >= p->ndim && p->n[d] != 1) return FRKC2_EINVAL;
  }
  if (cells(*p) > (size_t(1) << 34)) return FRKC2_EINVAL;
  if (!(p->dx > 0.0) || !std::isfinite(p->dx)) return FRKC2_EINVAL;
  if (p->kappa_kind == FRKC2_KAPPA_FIELD && !p->kappa) return FRKC2_EINVAL;
  if (p->kappa_kind == FRKC2_KAPPA_POWER && !(p->kappa_p > 0.0)) return FRKC2_EINVAL;
  if (p->precision == FRKC2_DFLOAT && (p->ndim != 2 || p->kappa_kind == FRKC2_KAPPA_POWER))
    return FRKC2_EUNSUPPORTED;  // the float-pair state has a 2D fixed-conductivity pass only
  return FRKC2_OK;
}

}  // namespace frkc2

using namespace frkc2;

extern "C" {

long long frkc2_launch_count(void) {
  const long long v = g_launches;
  g_launches = 0;
  return v;
}

frkc2_status frkc2_workspace_size(const frkc2_problem* prob, const frkc2_tuning* tune,
                                  size_t* bytes) {
  (void)tune;
  if (!bytes) return FRKC2_EINVAL;
  const frkc2_status v = validate_problem(prob);
  if (v != FRKC2_OK) return v;
  *bytes = step_layout(*prob).total;
  return FRKC2_OK;
}

frkc2_status frkc2_workspace_reset(void* ws, void* stream) {
  if (!ws) return FRKC2_EINVAL;
  return cudaMemsetAsync(ws, 0, 256, static_cast<cudaStream_t>(stream)) == cudaSuccess ? FRKC2_OK
                                                                                       : FRKC2_ECUDA;
}

frkc2_status frkc2_workspace_status(const void* ws, void* stream) {
  if (!ws) return FRKC2_EINVAL;
  unsigned st = 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(&st, ws, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return FRKC2_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return FRKC2_ECUDA;
  if (st & ST_BOUNDS) return FRKC2_EBOUNDS;
  if (st & ST_NONFINITE) return FRKC2_ENONFINITE;
  if (st & ST_TIMEOUT) return FRKC2_ETIMEOUT;
  return FRKC2_OK;
}

frkc2_status frkc2_rho_bound(const frkc2_problem* prob, const void* u, double* rho_dev,
                             void* stream) {
  const frkc2_status v = validate_problem(prob);
  if (v != FRKC2_OK) return v;
  if (!rho_dev || (reinterpret_cast<uintptr_t>(rho_dev) & 7)) return FRKC2_EINVAL;
  if (prob->kappa_kind == FRKC2_KAPPA_POWER && !u) return FRKC2_EINVAL;
  return launch_rho(*prob, u, rho_dev, static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? FRKC2_OK
             : FRKC2_ECUDA;
}

frkc2_status frkc2_step(frkc2_plan_t plan, const frkc2_problem* prob, double dt, int nsteps,
                        double rho, void* u, void* ws, size_t ws_bytes,
                        const frkc2_tuning* tune, void* stream) {
  if (!plan || !u || !ws || nsteps < 0) return FRKC2_EINVAL;
  const frkc2_status v = validate_problem(prob);
  if (v != FRKC2_OK) return v;
  if (!(dt > 0.0) || !std::isfinite(dt)) return FRKC2_EINVAL;
  if (reinterpret_cast<uintptr_t>(ws) & 255) return FRKC2_EINVAL;
  if (reinterpret_cast<uintptr_t>(u) & (state_bytes(prob->precision) - 1)) return FRKC2_EINVAL;
  if (rho > 0.0 && dt * rho > plan->beta * (1.0 + 1e-12)) return FRKC2_EUNSTABLE;
  const StepLayout L = step_layout(*prob);
  if (ws_bytes < L.total) return FRKC2_ENOMEM;
  const frkc2_problem& p = *prob;

  int k = (tune && tune->k) ? tune->k : default_k(p);
  if (tune && !tune->k && (tune->kernel == 2 || tune->kernel == 5)) k = 1;  // single-stage passes
  if (k < 1 || k > KMAX) return FRKC2_EINVAL;
  k = std::min(k, plan->s);
  int tx, ty, tz;
  default_tiles(p, k, &tx, &ty, &tz);
  if (tune && tune->tile_x) tx = tune->tile_x;
  if (tune && tune->tile_y) ty = tune->tile_y;
  if (tune && tune->tile_z) tz = tune->tile_z;
  if (p.ndim < 2) ty = 1;
  if (p.ndim < 3) tz = 1;
  if (tx < 1 || ty < 1 || tz < 1) return FRKC2_EINVAL;
  const int kern = tune ? tune->kernel : 0;
  if (kern < 0 || kern > 7) return FRKC2_EINVAL;
  const bool stream_ok = p.ndim == 2 && p.kappa_kind != FRKC2_KAPPA_POWER && k == 1;
  const bool tb_ok = tb2d_supported(p, k);
  const bool paired_ok = plan->paired && p.ndim == 2 && p.kappa_kind != FRKC2_KAPPA_POWER;
  bool use_stream2d = false, use_tb = false, use_paired = false, use_stream3d = false, use_small1d = false;
  bool use_tb_df = false, use_wf = false;
  const bool dfloat = p.precision == FRKC2_DFLOAT;
  const bool wf_ok = wf2d_supported(p, k, plan->s, u);
  const bool stream3d_ok = p.ndim == 3 && k == 1;
  const bool small1d_ok = small1d_supported(p, plan->s);
  if (kern == 6) {
    if (!small1d_ok) return FRKC2_EUNSUPPORTED;
    use_small1d = true;
  } else if (kern == 0 && small1d_ok && !(tune && tune->k)) {
    use_small1d = true;
  } else if (kern == 5) {
    if (!stream3d_ok) return FRKC2_EUNSUPPORTED;
    use_stream3d = true;
  } else if (dfloat) {
    // k = 1: the streaming pass; k > 1: the register-tiled pass (float-pair regions)
    if (kern == 1 || kern > 3 || (kern == 2 && k != 1) || 2 * k >= 64) return FRKC2_EUNSUPPORTED;
    if (kern == 3 || (kern == 0 && k > 1))
      use_tb_df = true;
    else
      use_stream2d = true;
  } else if (kern == 4) {
    if (!paired_ok) return FRKC2_EUNSUPPORTED;
    use_paired = true;
  } else if (kern == 0 && paired_ok && !(tune && tune->k)) {
    use_paired = true;
  } else if (kern == 2) {
    if (!stream_ok) return FRKC2_EUNSUPPORTED;
    use_stream2d = true;
  } else if (kern == 3) {
    if (!tb_ok) return FRKC2_EUNSUPPORTED;
    use_tb = true;
  } else if (kern == 7) {
    if (!wf_ok) return FRKC2_EUNSUPPORTED;
    use_wf = true;
  } else if (kern == 0) {
    // FP32 k-stage passes: the wavefront where it recomputes fewer cells than the 64 x 64 regions,
    // allowing for its 8 % higher cost per computed cell-stage (measured at 2048^2, k = 8)
    bool wf_wins = false;
    if (wf_ok && tb_ok && k > 1) {
      const int T = 64 - 2 * k, nx = int(p.n[0]), ny = int(p.n[1]);
      const double regions = double((nx + T - 1) / T) * ((ny + T - 1) / T) * 64.0 * 64.0 / (double(nx) * ny);
      wf_wins = 1.08 * wf2d_recompute(nx, ny, k) < regions;
    }
    if (wf_wins || (wf_ok && !tb_ok && k > 1))
      use_wf = true;
    else if (tb_ok && k > 1)
      use_tb = true;
    else if (stream3d_ok)
      use_stream3d = true;
    else
      use_stream2d = stream_ok;
  }
  if (use_stream2d && !(tune && tune->tile_y)) ty = 64;
  {
    PassArgs probe{};
    probe.tx = tx;
    probe.ty = ty;
    probe.tz = tz;
    probe.hx = k;
    probe.hy = p.ndim >= 2 ? k : 0;
    probe.hz = p.ndim >= 3 ? k : 0;
    if (!use_stream2d && !use_tb && !use_paired && !use_stream3d && !use_small1d && !use_tb_df && !use_wf &&
        generic_smem_bytes(p, probe) > size_t(smem_optin()))
      return FRKC2_EINVAL;
  }
  if (nsteps == 0) return FRKC2_OK;
  const NvtxRange call_range("frkc2_step");

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(ws);
  if (p.kappa_kind != FRKC2_KAPPA_POWER) {
    if (launch_faces(p, base + L.fx, base + L.fy, base + L.fz, st) != cudaSuccess) return FRKC2_ECUDA;
  }
  void* ua = base + L.ua;
  void* ub = base + L.ub;
  void* va = base + L.va;
  void* vb = base + L.vb;
  const int s = plan->s;
  const int npass = (s + k - 1) / k;
  const double h2 = p.dx * p.dx;

  PassArgs a{};
  a.ndim = p.ndim;
  a.bc = p.bc;
  a.nx = int(p.n[0]);
  a.ny = int(p.n[1]);
  a.nz = int(p.n[2]);
  a.tx = tx;
  a.ty = ty;
  a.tz = tz;
  a.fx = base + L.fx;
  a.fy = base + L.fy;
  a.fz = base + L.fz;
  a.kc = p.kappa_c;
  a.kp = p.kappa_p;
  a.status = reinterpret_cast<unsigned*>(base + L.status);

  if (use_small1d) {  // the whole job in one cluster launch
    // kernel 6: CTAs in the cluster, stages per halo exchange, threads per CTA (0: library choice)
    const int cl = tune ? tune->tile_x : 0, kx = tune ? tune->k : 0, th = tune ? tune->tile_y : 0;
    const cudaError_t e = launch_small1d(p, *plan, dt, nsteps, u, base + L.fx, a.status, st, cl, kx, th);
    return e == cudaSuccess ? FRKC2_OK : e == cudaErrorInvalidValue ? FRKC2_EINVAL : FRKC2_ECUDA;
  }
  const void* curU = u;
  const void* curV = nullptr;
  if (use_paired) {
    // real state throughout; each pass applies one conjugate pair (stages 2q, 2q+1)
    if (launch_face_pairs(p, base + L.fx, base + L.fy, base + L.fen, st) != cudaSuccess) return FRKC2_ECUDA;
    const int npair = s / 2;
    for (int n = 0; n < nsteps; ++n) {
      const NvtxRange step_range("frkc2 step");
      for (int q = 0; q < npair; ++q) {
        const NvtxRange pass_range("frkc2 pass");
        const bool last = n == nsteps - 1 && q == npair - 1;
        void* out = (last && curU != u) ? u : (curU == ua ? ub : ua);
        const double al = plan->a_re[2 * q], be = plan->a_im[2 * q];
        a.U_in = curU;
        a.U_out = out;
        a.V_in = a.V_out = nullptr;
        a.check_finite = q == npair - 1;
        a.ca[0] = dt * al / h2;
        a.ca[1] = dt * (al - be * be / al) / h2;
        a.cb[0] = dt * ((al * al + be * be) / al) / h2;
        if (launch_pass_paired2d(p, a, base + L.fen, st) != cudaSuccess) return FRKC2_ECUDA;
        curU = out;
      }
    }
    if (curU != u &&
        cudaMemcpyAsync(u, curU, cells(p) * state_bytes(p.precision), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return FRKC2_ECUDA;
    return FRKC2_OK;
  }
  if (use_tb_df) {
    // float-pair state (float4 per cell) between passes, in the ua (with va) and ub (with vb) slots
    // a pass never writes the array it reads (its regions' halos overlap other CTAs' output
    // tiles): with one pass per step the real state alternates between u and ua
    for (int n = 0; n < nsteps; ++n) {
      const NvtxRange step_range("frkc2 step");
      for (int q = 0; q < npass; ++q) {
        const NvtxRange pass_range("frkc2 pass");
        const int l0 = q * k, kq = std::min(k, s - l0);
        const bool first = q == 0, last = q == npass - 1;
        void* outW = (curU == ua) ? ub : ua;
        void* outU = last && curU != u ? u : outW;
        a.k = kq;
        a.U_in = curU;
        a.V_in = nullptr;
        a.in_mode = first ? PASS_IO_REAL : PASS_IO_COMPLEX;
        a.U_out = outU;
        a.V_out = nullptr;
        a.out_mode = last ? PASS_IO_REAL : PASS_IO_COMPLEX;
        a.check_finite = last ? 1 : 0;
        for (int j = 0; j < kq; ++j) {
          a.ca[j] = dt * plan->a_re[l0 + j] / h2;
          a.cb[j] = dt * plan->a_im[l0 + j] / h2;
          a.caf[j] = float(a.ca[j]);
          a.cbf[j] = float(a.cb[j]);
        }
        if (launch_pass_tb2d_df(p, a, st, n > 0 || q > 0) != cudaSuccess) return FRKC2_ECUDA;
        curU = outU;
      }
    }
    if (curU != u &&
        cudaMemcpyAsync(u, curU, cells(p) * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return FRKC2_ECUDA;
    return FRKC2_OK;
  }
  if (use_wf) {
    // interleaved (U, V) float2 state between passes in the ua (with va) and ub (with vb) slots;
    // a step's first pass reads the real state, its last writes it.  A pass never writes the
    // array it reads (a strip's halo columns and a chunk's first rows are other CTAs' output):
    // with one pass per step the real state alternates between u and ua.
    if (launch_faces_wf(p, base + L.fx, base + L.fy, base + L.fen, st) != cudaSuccess) return FRKC2_ECUDA;
    const int chunk_rows = tune ? tune->tile_y : 0;
    for (int n = 0; n < nsteps; ++n) {
      const NvtxRange step_range("frkc2 step");
      for (int q = 0; q < npass; ++q) {
        const NvtxRange pass_range("frkc2 pass");
        const int l0 = q * k, kq = std::min(k, s - l0);
        const bool first = q == 0, last = q == npass - 1;
        void* outW = (curU == ua) ? ub : ua;
        void* outU = last && curU != u ? u : outW;
        a.k = kq;
        a.U_in = curU;
        a.V_in = nullptr;
        a.U_out = outU;
        a.V_out = nullptr;
        a.check_finite = last ? 1 : 0;
        for (int j = 0; j < kq; ++j) {
          a.caf[j] = float(dt * plan->a_re[l0 + j] / h2);
          a.cbf[j] = float(dt * plan->a_im[l0 + j] / h2);
        }
        if (launch_pass_wf2d(p, a, base + L.fen, chunk_rows, first, last, st, n > 0 || q > 0,
                             tune ? tune->wait_limit : 0, tune && n == 0 && q == 0 ? tune->fault_inject : 0) !=
            cudaSuccess)
          return FRKC2_ECUDA;
        curU = outU;
      }
    }
    if (curU != u &&
        cudaMemcpyAsync(u, curU, cells(p) * sizeof(float), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return FRKC2_ECUDA;
    return FRKC2_OK;
  }
  if (use_stream2d) {
    // interleaved complex state between passes: W buffers at ua (with va) and ub (with vb)
    if (launch_face_pairs(p, base + L.fx, base + L.fy, base + L.fen, st) != cudaSuccess) return FRKC2_ECUDA;
    a.k = 1;
    a.hx = a.hy = 1;
    a.hz = 0;
    for (int n = 0; n < nsteps; ++n) {
      const NvtxRange step_range("frkc2 step");
      for (int l = 0; l < s; ++l) {
        const NvtxRange pass_range("frkc2 pass");
        const bool first = l == 0, last = l == s - 1;
        a.U_in = first ? u : curU;
        a.V_in = nullptr;
        a.in_mode = first ? PASS_IO_REAL : PASS_IO_COMPLEX;
        void* outW = (curU == ua) ? ub : ua;
        a.U_out = last ? u : outW;
        a.V_out = nullptr;
        a.out_mode = last ? PASS_IO_REAL : PASS_IO_COMPLEX;
        a.check_finite = last ? 1 : 0;
        a.ca[0] = dt * plan->a_re[l] / h2;
        a.cb[0] = dt * plan->a_im[l] / h2;
        a.caf[0] = float(a.ca[0]);
        a.cbf[0] = float(a.cb[0]);
        const cudaError_t e = dfloat ? launch_pass_stream2d_df(p, a, base + L.fen, st)
                                     : launch_pass_stream2d(p, a, base + L.fen, st);
        if (e != cudaSuccess) return FRKC2_ECUDA;
        curU = last ? u : outW;
      }
    }
    return FRKC2_OK;
  }
  for (int n = 0; n < nsteps; ++n) {
      const NvtxRange step_range("frkc2 step");
    for (int q = 0; q < npass; ++q) {
      const NvtxRange pass_range("frkc2 pass");
      const int l0 = q * k;
      const int kq = std::min(k, s - l0);
      const bool last = q == npass - 1;
      void* outU;
      if (last && curU != u)
        outU = u;
      else
        outU = (curU == ua) ? ub : ua;
      void* outV = last ? nullptr : (curV == va ? vb : va);
      a.k = kq;
      a.hx = kq;
      a.hy = p.ndim >= 2 ? kq : 0;
      a.hz = p.ndim >= 3 ? kq : 0;
      a.U_in = curU;
      a.V_in = curV;
      a.U_out = outU;
      a.V_out = outV;
      a.check_finite = last ? 1 : 0;
      for (int j = 0; j < kq; ++j) {
        a.ca[j] = dt * plan->a_re[l0 + j] / h2;
        a.cb[j] = dt * plan->a_im[l0 + j] / h2;
        a.caf[j] = float(a.ca[j]);
        a.cbf[j] = float(a.cb[j]);
      }
      a.in_mode = curV ? PASS_IO_PLANAR : PASS_IO_REAL;
      a.out_mode = outV ? PASS_IO_PLANAR : PASS_IO_REAL;
      // passes after the first may start while the previous one drains (face conductivities,
      // written before the first pass, are read before the wait for the previous pass)
      const cudaError_t e = use_tb ? launch_pass_tb2d(p, a, st, n > 0 || q > 0)
                            : use_stream3d ? launch_pass_stream3d(p, a, st)
                                           : launch_pass_generic(p, a, st);
      if (e != cudaSuccess) return FRKC2_ECUDA;
      curU = outU;
      curV = outV;
    }
  }
  if (curU != u) {
    if (cudaMemcpyAsync(u, curU, cells(p) * state_bytes(p.precision), cudaMemcpyDeviceToDevice, st) !=
        cudaSuccess)
      return FRKC2_ECUDA;
  }
  return FRKC2_OK;
}

frkc2_status frkc2_adaptive_workspace_size(const frkc2_problem* prob, const frkc2_tuning* tune, size_t* bytes) {
  (void)tune;
  if (!bytes) return FRKC2_EINVAL;
  const frkc2_status v = validate_problem(prob);
  if (v != FRKC2_OK) return v;
  if (prob->precision == FRKC2_DFLOAT) return FRKC2_EUNSUPPORTED;
  const size_t N = cells(*prob), S = state_bytes(prob->precision);
  // step workspace + two embedded-solution buffers + the error sum
  *bytes = step_layout(*prob).total + 2 * align256(N * S) + 256;
  return FRKC2_OK;
}

frkc2_status frkc2_step_adaptive(frkc2_plan_t plan, const frkc2_problem* prob, double t_end, double tol,
                                 double dt0, double rho, void* u, void* ws, size_t ws_bytes,
                                 const frkc2_tuning* tune, frkc2_adaptive_stats* stats, void* stream) {
  const frkc2::NvtxRange call_range("frkc2_step_adaptive");
  if (!plan || !u || !ws || !(t_end > 0.0) || !(tol > 0.0) || !(dt0 > 0.0)) return FRKC2_EINVAL;
  const frkc2_status v = validate_problem(prob);
  if (v != FRKC2_OK) return v;
  if (prob->precision == FRKC2_DFLOAT) return FRKC2_EUNSUPPORTED;
  if (reinterpret_cast<uintptr_t>(ws) & 255) return FRKC2_EINVAL;
  size_t need = 0;
  frkc2_adaptive_workspace_size(prob, tune, &need);
  if (ws_bytes < need) return FRKC2_ENOMEM;
  const frkc2_problem& p = *prob;
  const StepLayout L = step_layout(p);
  const size_t N = cells(p), SB = state_bytes(p.precision);
  char* base = static_cast<char*>(ws);
  char* hA = base + L.total;
  char* hB = hA + align256(N * SB);
  double* esum = reinterpret_cast<double*>(hB + align256(N * SB));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int k = (tune && tune->k) ? tune->k : default_k(p);
  if (k < 1 || k > KMAX) return FRKC2_EINVAL;
  k = std::min(k, plan->s);
  int tx, ty, tz;
  default_tiles(p, k, &tx, &ty, &tz);
  if (tune && tune->tile_x) tx = tune->tile_x;
  if (tune && tune->tile_y) ty = tune->tile_y;
  if (tune && tune->tile_z) tz = tune->tile_z;
  if (p.ndim < 2) ty = 1;
  if (p.ndim < 3) tz = 1;
  if (p.kappa_kind != FRKC2_KAPPA_POWER &&
      launch_faces(p, base + L.fx, base + L.fy, base + L.fz, st) != cudaSuccess)
    return FRKC2_ECUDA;
  PassArgs a{};
  a.ndim = p.ndim;
  a.bc = p.bc;
  a.nx = int(p.n[0]);
  a.ny = int(p.n[1]);
  a.nz = int(p.n[2]);
  a.tx = tx;
  a.ty = ty;
  a.tz = tz;
  a.fx = base + L.fx;
  a.fy = base + L.fy;
  a.fz = base + L.fz;
  a.kc = p.kappa_c;
  a.kp = p.kappa_p;
  a.status = reinterpret_cast<unsigned*>(base + L.status);
  // 2D fixed conductivity: the streaming pass (one stage a launch, interleaved complex state
  // in the ua / ub slots, the embedded solution advanced alongside); otherwise the tile pass
  const bool streamed = p.ndim == 2 && p.kappa_kind != FRKC2_KAPPA_POWER && p.precision != FRKC2_DFLOAT &&
                        !(tune && (tune->kernel != 0 || tune->k > 1 || tune->tile_x || tune->tile_y));
  if (!streamed) {  // only the tile pass needs shared memory for a tile of k stages
    PassArgs probe = a;
    probe.hx = k;
    probe.hy = p.ndim >= 2 ? k : 0;
    probe.hz = p.ndim >= 3 ? k : 0;
    probe.H_out = hA;
    if (generic_smem_bytes(p, probe) > size_t(smem_optin())) return FRKC2_EINVAL;
  }
  void* UA = base + L.ua;
  void* VA = base + L.va;
  void* UB = base + L.ub;
  void* VB = base + L.vb;
  if (streamed && launch_face_pairs(p, base + L.fx, base + L.fy, base + L.fen, st) != cudaSuccess)
    return FRKC2_ECUDA;
  const int s = plan->s, npass = (s + k - 1) / k;
  const double h2 = p.dx * p.dx, safe = 0.8, tmax = rho > 0.0 ? plan->beta / rho : 0.0;
  double t = 0.0, T = dt0, T_prev = 0.0, e_prev = 0.0;
  int acc = 0, rej = 0;
  const int max_attempts = 1000000;
  while (t < t_end * (1.0 - 1e-14) && acc + rej < max_attempts) {
    T = std::min(T, t_end - t);
    if (tmax > 0.0) T = std::min(T, tmax);
    // one step from u into the ping-pong buffers; the embedded solution alongside
    const void* cU = u;
    const void* cV = nullptr;
    const void* cH = u;
    for (int l = 0; streamed && l < s; ++l) {
      const bool first = l == 0, last = l == s - 1;
      void* oW = (cU == UA) ? UB : UA;  // the step's result stays off u until it is accepted
      void* oH = (cH == hA) ? hB : hA;
      a.U_in = cU;
      a.V_in = nullptr;
      a.in_mode = first ? PASS_IO_REAL : PASS_IO_COMPLEX;
      a.U_out = oW;
      a.V_out = nullptr;
      a.out_mode = last ? PASS_IO_REAL : PASS_IO_COMPLEX;
      a.H_in = cH;
      a.H_out = oH;
      a.check_finite = 0;
      a.ca[0] = T * plan->a_re[l] / h2;
      a.cb[0] = T * plan->a_im[l] / h2;
      if (launch_pass_stream2d(p, a, base + L.fen, st) != cudaSuccess) return FRKC2_ECUDA;
      cU = oW;
      cH = oH;
    }
    for (int q = 0; !streamed && q < npass; ++q) {
      const int l0 = q * k, kq = std::min(k, s - l0);
      const bool last = q == npass - 1;
      void* oU = (cU == UA) ? UB : UA;
      void* oV = last ? nullptr : ((cV == VA) ? VB : VA);
      void* oH = (cH == hA) ? hB : hA;
      a.k = kq;
      a.hx = kq;
      a.hy = p.ndim >= 2 ? kq : 0;
      a.hz = p.ndim >= 3 ? kq : 0;
      a.U_in = cU;
      a.V_in = cV;
      a.H_in = cH;
      a.U_out = oU;
      a.V_out = oV;
      a.H_out = oH;
      a.check_finite = 0;
      for (int j = 0; j < kq; ++j) {
        a.ca[j] = T * plan->a_re[l0 + j] / h2;
        a.cb[j] = T * plan->a_im[l0 + j] / h2;
      }
      if (launch_pass_generic(p, a, st) != cudaSuccess) return FRKC2_ECUDA;
      cU = oU;
      cV = oV;
      cH = oH;
    }
    if (launch_err_sum(p, cU, cH, esum, st) != cudaSuccess) return FRKC2_ECUDA;
    double e2 = 0.0;
    if (cudaMemcpyAsync(&e2, esum, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return FRKC2_ECUDA;
    double e = std::sqrt(e2 / double(N)) / tol;  // Eq. 15, root mean square over the cells
    if (!std::isfinite(e) || e > 1.0) {
      ++rej;
      T *= safe / std::sqrt(std::isfinite(e) ? e : 1e10);
      continue;
    }
    if (cudaMemcpyAsync(u, cU, N * SB, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return FRKC2_ECUDA;
    ++acc;
    t += T;
    e = std::max(e, 1e-10);
    double fac = safe / std::sqrt(e);
    if (T_prev > 0.0) fac *= (T / T_prev) * std::sqrt(e_prev / e);  // Eq. 16
    if (stats) {
      stats->dt_last = T;
      stats->err_last = e;
    }
    T_prev = T;
    e_prev = e;
    T *= std::min(fac, 5.0);
  }
  if (stats) {
    stats->accepted = acc;
    stats->rejected = rej;
    stats->t = t;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return FRKC2_ECUDA;
  return t >= t_end * (1.0 - 1e-14) ? FRKC2_OK : FRKC2_ETIMEOUT;
}

}  // extern "C"
