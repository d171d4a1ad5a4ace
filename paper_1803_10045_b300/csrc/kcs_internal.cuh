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
struct AngleTab {
  float beta;      // d fr / d bin
  float gamma;     // d fr / d major step
  float w;         // step weight h / max(|cos|, |sin|)
  int xmajor;      // 1: major axis = columns
  float inv_beta;  // 1 / beta (only to bound candidate bins; exact tests use beta)
  float pad[3];
};

}  // namespace kcs

struct kcs_geometry {
  int nx, ny, nz, B, A, S;
  float vox, bin;
  int device;
  kcs::AngleTab* d_ang;   // [A]
  int* d_angles;          // subset lists concatenated, then 0..A-1 at offset A
  std::vector<int> h_angles;
  std::vector<int> off;   // off[k] .. off[k+1]: angles of subset k
  int max_sub;
};

namespace kcs {

inline int subset_count(const kcs_geometry* g, int k) {
  return k < 0 ? g->A : g->off[k + 1] - g->off[k];
}
inline const int* subset_dev(const kcs_geometry* g, int k) {
  return k < 0 ? g->d_angles + g->A : g->d_angles + g->off[k];
}
inline size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

// ------------------------------------------------------------ kinetics
// Each a-dependent channel is e^{-aD} sum_n a^n c_n with c_n >= 0.  The series
// is tabulated around NCENT expansion centres a0 = c * DCENT (Taylor shift of the
// float64 base series, again non-negative coefficients), so a voxel sums at most
// 8 terms (intervals <= 5 min, delta = a - a0 in [0, 1/16)) whatever a is; the
// centre spacing trades table size (60 centres, 0.8 MB for 24 intervals) for
// series length (1/4 spacing needed up to 13 terms).  Table layout
// [interval][term][part][centre] (part = 4 channels): the lanes of a warp, each
// on its own centre, read one short contiguous run per load.
constexpr int NB = 128;         // base terms tabulated in float64
#ifndef KCS_CENT_PER_UNIT
#define KCS_CENT_PER_UNIT 16
#endif
#ifndef KCS_KC
#define KCS_KC 10
#endif
constexpr int KC = KCS_KC;                       // terms per centre
constexpr int NCENT = 15 * KCS_CENT_PER_UNIT / 4;   // valid for 0 <= a < NCENT * DCENT
constexpr float DCENT = 1.0f / KCS_CENT_PER_UNIT;
constexpr int NCH = 12;         // channels per term, padded to 3 float4
constexpr double DT_MAX = 5.0;  // longest propagation interval (min)

// Channel numbering of the float64 base series.
enum { CH_M1 = 0, CH_G, CH_M2, CH_H, CH_M3, CH_D1, CH_GP, CH_D2, CH_HP, CH_D3 };
// Packing of a term's channels into 3 float4 parts: part 0 (m1, m2, m3, d1) and
// part 1 (d2, d3, -, -) depend on the input over the interval; part 2
// (g, h, gp, hp) only on a and D, so it is evaluated once per distinct D.
__host__ __device__ constexpr int ch_slot(int ch) {
  return ch == CH_M1 ? 0 : ch == CH_M2 ? 1 : ch == CH_M3 ? 2 : ch == CH_D1 ? 3
       : ch == CH_D2 ? 4 : ch == CH_D3 ? 5
       : ch == CH_G ? 8 : ch == CH_H ? 9 : ch == CH_GP ? 10 : 11;   // CH_HP
}

struct KinDev {
  const float4* coef;   // [n_iv][KC][3][NCENT] float4 (12 channels = 3 parts)
  const float* iv_dt;   // [n_iv] interval length (min)
  const int* iv_code;   // [n_iv]: -1 gap, else 2*frame + (last piece of the frame)
  const float* fr_cp;   // [M] frame average of Cp
  const float* fr_inv;  // [M] 1 / frame duration
  int n_iv;
  int M;
};

}  // namespace kcs

struct kcs_kinetics {
  int M;
  int n_iv;
  int device;
  float4* d_coef;
  float* d_iv_dt;
  int* d_iv_code;
  float* d_fr_cp;
  float* d_fr_inv;
  double* d_tmp;   // per-interval doubles used while tabulating
  double* d_base;  // [n_iv][NB][10] float64 base series
  kcs::KinDev dev() const {
    return kcs::KinDev{d_coef, d_iv_dt, d_iv_code, d_fr_cp, d_fr_inv, n_iv, M};
  }
};

namespace kcs {
// launchers shared between translation units
int launch_tac_eval(const kcs_kinetics* k, int64_t n_vox, const float* params, float* F,
                    float* J, cudaStream_t s);
}  // namespace kcs
