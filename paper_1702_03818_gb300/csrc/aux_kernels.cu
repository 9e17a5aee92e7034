// Per-step set-up kernels: face conductivities and the Gershgorin spectral-radius bound.
#include <cuda_runtime.h>

#include "frkc2_internal.h"

namespace frkc2 {
namespace {

struct FaceArgs {
  int ndim, bc, kind;
  int nx, ny, nz;
  double c;
  const void* kappa;
  void* fx;
  void* fy;
  void* fz;
};

// Face i along an axis lies between cells i-1 and i (i = 0..n).  Interior faces take the
// arithmetic mean of their two cells; periodic faces 0 and n are the same wrap face; a
// Dirichlet boundary face takes its interior cell's value.
template <class A>
__device__ __forceinline__ A face_value(const A* K, int i, int n, size_t base, size_t stride,
                                        bool periodic) {
  if (periodic) {
    const int lo = (i == 0 || i == n) ? n - 1 : i - 1;
    const int hi = (i == n) ? 0 : i;
    return A(0.5) * (K[base + size_t(lo) * stride] + K[base + size_t(hi) * stride]);
  }
  if (i == 0) return A(0.5) * (K[base] + K[base]);
  if (i == n) return A(0.5) * (K[base + size_t(n - 1) * stride] + K[base + size_t(n - 1) * stride]);
  return A(0.5) * (K[base + size_t(i - 1) * stride] + K[base + size_t(i) * stride]);
}

template <class A>
__global__ void k_faces(const FaceArgs a) {
  const A* K = static_cast<const A*>(a.kappa);
  const bool periodic = a.bc == FRKC2_BC_PERIODIC;
  const bool cst = a.kind == FRKC2_KAPPA_CONST;
  const size_t nfx = size_t(a.nz) * a.ny * (a.nx + 1);
  const size_t nfy = a.ndim >= 2 ? size_t(a.nz) * (a.ny + 1) * a.nx : 0;
  const size_t nfz = a.ndim >= 3 ? size_t(a.nz + 1) * a.ny * a.nx : 0;
  const size_t total = nfx + nfy + nfz;
  for (size_t t = blockIdx.x * size_t(blockDim.x) + threadIdx.x; t < total;
       t += size_t(gridDim.x) * blockDim.x) {
    if (t < nfx) {
      const int i = int(t % (a.nx + 1));
      const size_t row = t / (a.nx + 1);  // z*ny + y
      static_cast<A*>(a.fx)[t] = cst ? A(a.c) : face_value<A>(K, i, a.nx, row * a.nx, 1, periodic);
    } else if (t < nfx + nfy) {
      const size_t q = t - nfx;
      const int x = int(q % a.nx);
      const size_t r = q / a.nx;
      const int j = int(r % (a.ny + 1));
      const int z = int(r / (a.ny + 1));
      static_cast<A*>(a.fy)[q] =
          cst ? A(a.c) : face_value<A>(K, j, a.ny, size_t(z) * a.ny * a.nx + x, size_t(a.nx), periodic);
    } else {
      const size_t q = t - nfx - nfy;
      const size_t plane = size_t(a.ny) * a.nx;
      const int kz = int(q / plane);
      const size_t xy = q % plane;
      static_cast<A*>(a.fz)[q] = cst ? A(a.c) : face_value<A>(K, kz, a.nz, xy, plane, periodic);
    }
  }
}

struct RhoArgs {
  int ndim, bc, kind;
  int nx, ny, nz;
  double c, p, dx;
  const void* field;   // kappa (FIELD) or u (POWER)
  double* out;
};

template <class T>
__device__ __forceinline__ double cell_kappa_real(const RhoArgs& a, const T* F, size_t g) {
  if (a.kind == FRKC2_KAPPA_CONST) return a.c;
  if (a.kind == FRKC2_KAPPA_FIELD) return double(F[g]);
  return __dadd_rn(1.0, __dmul_rn(a.c, pow(double(F[g]), a.p)));
}

// rho = max_c (2 acc_c)/(dx*dx), acc_c = sum of face values (kappa_c + kappa_nb)/2, x axis
// first, low face first.  Halving and doubling are exact, so 2 acc_c equals the same running
// sum of the unhalved pair sums (kappa_c + kappa_nb); and rounding is monotonic, so the
// maximum may be taken before the one division by dx*dx, done once per block.
// Each warp takes whole rows (fixed y, z) and its lanes walk x, so no index is divided.
template <class T>
__global__ void k_rho(const RhoArgs a) {
  const T* F = static_cast<const T*>(a.field);
  const bool periodic = a.bc == FRKC2_BC_PERIODIC;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const size_t sy = size_t(nx), sz = size_t(nx) * ny;
  const double h2 = __dmul_rn(a.dx, a.dx);
  const int lane = threadIdx.x & 31;
  const long long warp = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  const long long rows = (long long)ny * nz;
  // the neighbour's conductivity, or the ghost value when it lies outside a Dirichlet grid
  auto nb = [&](double kc, size_t g, int c, int n, size_t stride, int side) -> double {
    const int q = side ? c + 1 : c - 1;
    if (q >= 0 && q < n) return cell_kappa_real<T>(a, F, side ? g + stride : g - stride);
    if (periodic) return cell_kappa_real<T>(a, F, side ? g - size_t(n - 1) * stride : g + size_t(n - 1) * stride);
    return a.kind == FRKC2_KAPPA_POWER ? 1.0 : kc;
  };
  double best2 = 0.0;  // max of 2 acc_c
  for (long long r = warp; r < rows; r += nwarps) {
    const int y = int(r % ny), z = int(r / ny);
    const size_t row0 = size_t(r) * nx;
    for (int x = lane; x < nx; x += 32) {
      const size_t g = row0 + x;
      const double kc = cell_kappa_real<T>(a, F, g);
      double acc2 = __dadd_rn(kc, nb(kc, g, x, nx, 1, 0));
      acc2 = __dadd_rn(acc2, __dadd_rn(kc, nb(kc, g, x, nx, 1, 1)));
      if (a.ndim >= 2) {
        acc2 = __dadd_rn(acc2, __dadd_rn(kc, nb(kc, g, y, ny, sy, 0)));
        acc2 = __dadd_rn(acc2, __dadd_rn(kc, nb(kc, g, y, ny, sy, 1)));
      }
      if (a.ndim >= 3) {
        acc2 = __dadd_rn(acc2, __dadd_rn(kc, nb(kc, g, z, nz, sz, 0)));
        acc2 = __dadd_rn(acc2, __dadd_rn(kc, nb(kc, g, z, nz, sz, 1)));
      }
      best2 = (acc2 > best2 || acc2 != acc2) ? acc2 : best2;
    }
  }
  // block max, then one atomic per block on the bit pattern (non-negative doubles, and NaN,
  // order like their bits read as unsigned integers)
  unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(best2));
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_xor_sync(0xffffffffu, bits, o);
    bits = other > bits ? other : bits;
  }
  __shared__ unsigned long long warp_best[32];
  const int w = threadIdx.x >> 5;
  if (lane == 0) warp_best[w] = bits;
  __syncthreads();
  if (w == 0) {
    bits = lane < int(blockDim.x >> 5) ? warp_best[lane] : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long other = __shfl_xor_sync(0xffffffffu, bits, o);
      bits = other > bits ? other : bits;
    }
    if (lane == 0) {
      const double v = __ddiv_rn(__longlong_as_double(static_cast<long long>(bits)), h2);
      atomicMax(reinterpret_cast<unsigned long long*>(a.out),
                static_cast<unsigned long long>(__double_as_longlong(v)));
    }
  }
}

int grid_for(size_t work, int threads) {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t need = (work + threads - 1) / threads;
  const size_t cap = size_t(sms) * 8;
  return int(need < cap ? (need ? need : 1) : cap);
}

}  // namespace

cudaError_t launch_faces(const frkc2_problem& p, void* fx, void* fy, void* fz, cudaStream_t st) {
  FaceArgs a{p.ndim, p.bc, p.kappa_kind, int(p.n[0]), int(p.n[1]), int(p.n[2]), p.kappa_c,
             p.kappa, fx, fy, fz};
  const FaceLayout L = faces_layout(p);
  const size_t total = L.nfx + L.nfy + L.nfz;
  const int threads = 256;
  if (p.precision == FRKC2_FP64)
    k_faces<double><<<grid_for(total, threads), threads, 0, st>>>(a);
  else
    k_faces<float><<<grid_for(total, threads), threads, 0, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_rho(const frkc2_problem& p, const void* u, double* rho_dev, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(rho_dev, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  RhoArgs a{p.ndim, p.bc, p.kappa_kind, int(p.n[0]), int(p.n[1]), int(p.n[2]), p.kappa_c,
            p.kappa_p, p.dx, p.kappa_kind == FRKC2_KAPPA_POWER ? u : p.kappa, rho_dev};
  const int threads = 256;
  // the field is read in the state precision for POWER and the kappa precision otherwise
  const bool dbl = p.kappa_kind == FRKC2_KAPPA_POWER ? state_bytes(p.precision) == 8
                                                     : arith_bytes(p.precision) == 8;
  if (dbl)
    k_rho<double><<<grid_for(size_t(p.n[1]) * p.n[2] * 32, threads), threads, 0, st>>>(a);
  else
    k_rho<float><<<grid_for(size_t(p.n[1]) * p.n[2] * 32, threads), threads, 0, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

}  // namespace frkc2
