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

// rho = max_c (2 acc_c)/(dx*dx), acc_c = sum of face values, x axis first, low face first.
template <class T>
__global__ void k_rho(const RhoArgs a) {
  const T* F = static_cast<const T*>(a.field);
  const bool periodic = a.bc == FRKC2_BC_PERIODIC;
  const size_t N = size_t(a.nx) * a.ny * a.nz;
  const double h2 = __dmul_rn(a.dx, a.dx);
  double best = 0.0;
  for (size_t g = blockIdx.x * size_t(blockDim.x) + threadIdx.x; g < N;
       g += size_t(gridDim.x) * blockDim.x) {
    const int x = int(g % a.nx);
    const int y = int((g / a.nx) % a.ny);
    const int z = int(g / (size_t(a.nx) * a.ny));
    const double kc = cell_kappa_real<T>(a, F, g);
    double acc = 0.0;
    const int n3[3] = {a.nx, a.ny, a.nz};
    const int c3[3] = {x, y, z};
    const size_t s3[3] = {1, size_t(a.nx), size_t(a.nx) * a.ny};
    for (int d = 0; d < a.ndim; ++d) {
      for (int side = 0; side < 2; ++side) {
        const int nbc = side ? c3[d] + 1 : c3[d] - 1;
        double kn;
        if (nbc >= 0 && nbc < n3[d]) {
          kn = cell_kappa_real<T>(a, F, side ? g + s3[d] : g - s3[d]);
        } else if (periodic) {
          const size_t gw = side ? g - size_t(n3[d] - 1) * s3[d] : g + size_t(n3[d] - 1) * s3[d];
          kn = cell_kappa_real<T>(a, F, gw);
        } else {
          kn = a.kind == FRKC2_KAPPA_POWER ? 1.0 : kc;
        }
        acc = __dadd_rn(acc, __dmul_rn(0.5, __dadd_rn(kc, kn)));
      }
    }
    const double v = __ddiv_rn(__dmul_rn(2.0, acc), h2);
    best = (v > best || v != v) ? v : best;
  }
  // block max, then one atomic per block on the bit pattern (non-negative doubles, and NaN,
  // order like their bits read as unsigned integers)
  unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(best));
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_xor_sync(0xffffffffu, bits, o);
    bits = other > bits ? other : bits;
  }
  __shared__ unsigned long long warp_best[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) warp_best[w] = bits;
  __syncthreads();
  if (w == 0) {
    bits = lane < int(blockDim.x >> 5) ? warp_best[lane] : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long other = __shfl_xor_sync(0xffffffffu, bits, o);
      bits = other > bits ? other : bits;
    }
    if (lane == 0) atomicMax(reinterpret_cast<unsigned long long*>(a.out), bits);
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
  const size_t N = cells(p);
  const int threads = 256;
  // the field is read in the state precision for POWER and the kappa precision otherwise
  const bool dbl = p.kappa_kind == FRKC2_KAPPA_POWER ? state_bytes(p.precision) == 8
                                                     : arith_bytes(p.precision) == 8;
  if (dbl)
    k_rho<double><<<grid_for(N, threads), threads, 0, st>>>(a);
  else
    k_rho<float><<<grid_for(N, threads), threads, 0, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

}  // namespace frkc2
