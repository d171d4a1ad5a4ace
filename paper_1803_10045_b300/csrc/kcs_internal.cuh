// Internal declarations of the kcs library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/kcs.h"

namespace kcs {

// ------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
void clear_error();

#define KCS_REQUIRE(cond, ...)                 \
  do {                                         \
    if (!(cond)) {                             \
      ::kcs::set_error(__VA_ARGS__);           \
      return KCS_ERR_INVALID_ARG;              \
    }                                          \
  } while (0)

#define KCS_CUDA(call)                                                              \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      ::kcs::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),      \
                       __FILE__, __LINE__);                                         \
      return e_ == cudaErrorMemoryAllocation ? KCS_ERR_OOM : KCS_ERR_CUDA;          \
    }                                                                               \
  } while (0)

// A launch error (bad configuration) is reported without synchronising.
#define KCS_LAUNCHED()                                                              \
  do {                                                                              \
    cudaError_t e_ = cudaGetLastError();                                            \
    if (e_ != cudaSuccess) {                                                        \
      ::kcs::set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_),  \
                       __FILE__, __LINE__);                                         \
      return KCS_ERR_CUDA;                                                          \
    }                                                                               \
  } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Scalar loads/stores of the storage types of the precision form.
__device__ __forceinline__ float ld1(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ld1(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ float ld1(const __half* p) { return __half2float(*p); }
__device__ __forceinline__ float ld1(const uint16_t* p) { return (float)*p; }
__device__ __forceinline__ void st1(float* p, float v) { *p = v; }
__device__ __forceinline__ void st1(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void st1(__half* p, float v) { *p = __float2half_rn(fminf(v, 65504.f)); }

// ------------------------------------------------------------ geometry
// Per-angle Joseph constants.  Along the major axis (index t, centred
// tf = t - (n_major-1)/2) the ray of bin b (centred bf = b - (B-1)/2) meets the
// fractional minor index fr = fma(bf, beta, fma(tf, gamma, (n_minor-1)/2)).
// x-major angles step over columns (minor = rows), the others over rows.
struct __align__(16) AngleTab {
  float beta;      // d fr / d bin
  float gamma;     // d fr / d major step
  float w;         // step weight h / max(|cos|, |sin|)
  int xmajor;      // 1: major axis = columns
  float inv_beta;  // 1 / beta (only to bound candidate bins; exact tests use beta)
  float tc;        // (n_major - 1) / 2: centre of the major axis
  float centre;    // (n_minor - 1) / 2: centre of the minor axis
  float rband;     // |1 / beta| + 1e-3: half-width in bins of the candidates of a voxel
  int pair;        // 1: at most two consecutive bins reach any voxel (see kcs_create_geometry)
  int pad_[3];     // spare; the back-projection's staged copy carries a block's row
                   // window (first row, row count) and the angle index here
};

}  // namespace kcs

struct kcs_geometry {
  int nx, ny, nz, B, A, S;
  float vox, bin;
  int device;
  kcs::AngleTab* d_ang;   // [A]
  int* d_angles;          // subset lists concatenated, then 0..A-1 at offset A
  std::vector<int> h_angles;
  std::vector<kcs::AngleTab> h_tab;   // host copy of d_ang (source of its asynchronous upload)
  std::vector<int> off;   // off[k] .. off[k+1]: angles of subset k
  int max_sub;
  int pair_all;           // every angle obeys the pair rule of the back-projection
};

namespace kcs {

inline int subset_count(const kcs_geometry* g, int k) {
  return k < 0 ? g->A : g->off[k + 1] - g->off[k];
}
inline const int* subset_dev(const kcs_geometry* g, int k) {
  return k < 0 ? g->d_angles + g->A : g->d_angles + g->off[k];
}
inline size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

// Division by a runtime divisor d >= 2 as one multiply-high.  With
// mul = ceil(2^32 / d) = (2^32 + e) / d, 0 <= e < d, the product n mul / 2^32
// equals n / d + n e / (d 2^32); for n (d - 1) < 2^32 the second term is below
// 1 / d, which cannot carry the fraction of n / d past the next integer, so
// __umulhi(n, mul) = floor(n / d) exactly.  The 64-bit form (mul = ceil(2^64 /
// d), __umul64hi) is exact for n (d - 1) < 2^64; d = 1 is encoded as mul = 0.
inline unsigned div_magic32(unsigned d) { return (unsigned)((0x100000000ull + d - 1) / d); }
inline unsigned long long div_magic64(unsigned long long d) {
  return d < 2 ? 0ull
               : (unsigned long long)((((unsigned __int128)1 << 64) + d - 1) / d);
}
__device__ __forceinline__ unsigned long long div64(unsigned long long n, unsigned long long mul) {
  return mul ? __umul64hi(n, mul) : n;
}

// ------------------------------------------------------------ kinetics
// The frame-integrated model is linear in K1, k3 and Vb once a = k2 + k3 is
// fixed:  F_m = (1 - Vb) K1 (A_m(a) + k3 B_m(a)) + Vb cp_m,  with A_m, B_m the
// frame averages of I = Cp * e^{-a t} and of its time integral.  A_m, B_m and
// their a-derivatives are tabulated in float64 on a uniform grid of a (NODES_
// PER_UNIT nodes per unit, 0 <= a <= A_MAX) once per frame schedule, from the
// input moments of every propagation interval (power series in a with
// non-negative coefficients, no cancellation near a -> 0 or a -> an input
// exponent).  Each grid cell holds, per frame, the coefficients of the cubic
// Hermite interpolants of A and B in the cell's local coordinate (formed in
// float64, rounded once): a voxel reads one aligned 32-byte entry per frame and
// evaluates A, B and their derivatives with a few fused multiply-adds.  Table
// layout [frame][cell], so the lanes of a warp (voxels with similar a) read
// neighbouring entries.
constexpr int NB = 128;                 // base terms of the input moments (float64)
constexpr double DT_MAX = 5.0;          // longest propagation interval (min)
constexpr int NODES_PER_UNIT = 512;     // grid spacing h = 1/512 in a (1/min)
constexpr double A_MAX = 3.75;          // tabulated range of a (the fit's box has a <= 3)
constexpr int N_NODES = (int)(A_MAX * NODES_PER_UNIT) + 2;
constexpr int N_CELLS = N_NODES - 1;

// Channel numbering of the float64 base series.
enum { CH_M1 = 0, CH_G, CH_M2, CH_H, CH_M3, CH_D1, CH_GP, CH_D2, CH_HP, CH_D3 };

struct KinDev {
  // [M][N_CELLS][2]: cubic coefficients (c0, c1, c2, c3) of A, then of B, on
  // cell c in s = a NODES_PER_UNIT - c:  A = c0 + s c1 + s^2 c2 + s^3 c3
  const float4* cell;
  const float* fr_cp;   // [M] frame average of Cp
  int M;
  unsigned div_m, div_4m;   // div_magic32(M), div_magic32(4 M)
};

}  // namespace kcs

struct kcs_kinetics {
  int M;
  int n_iv;
  int device;
  float4* d_cell;
  float* d_fr_cp;
  int* d_iv_code;
  double* d_tmp;   // per-interval doubles used while tabulating
  double* d_base;  // [n_iv][NB][10] float64 base series
  kcs::KinDev dev() const {
    return kcs::KinDev{d_cell, d_fr_cp, M, kcs::div_magic32((unsigned)M),
                       kcs::div_magic32(4u * (unsigned)M)};
  }
};

namespace kcs {
// launchers shared between translation units
int launch_tac_eval(const kcs_kinetics* k, int64_t n_vox, const float* params, float* F,
                    float* J, cudaStream_t s);
}  // namespace kcs
