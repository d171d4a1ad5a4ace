// Joseph projector, its exact transpose and the fused OS-MAP-OSL update
// (Eq. 2-3 of Scipioni et al., "Kinetic Compressive Sensing").
//
// Data layout: images [Z][ny][nx][M] and sinograms [Z][A][B][M] keep the M
// frames of one voxel / bin contiguous, so every sample of a ray moves whole
// float4 frame quads.  In the forward a warp holds 32/MQ rays, MQ = M/4 lanes
// each, so one load instruction fetches the contiguous frame vectors of several
// rays.  The back-projection is a gather: each voxel (one thread, all frames)
// recomputes the forward's sample positions with the same fused multiply-adds,
// so the set of (voxel, bin, weight) triples is exactly the forward's, with no
// atomics; the ratio rows of a voxel tile are staged in shared memory.

#include <cstdarg>
#include <cmath>
#include <algorithm>
#include <type_traits>

#include "kcs_internal.cuh"

namespace kcs {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
}
void clear_error() { g_err.clear(); }

// ------------------------------------------------------------ device helpers
__device__ __forceinline__ float4 f4(float v) { return make_float4(v, v, v, v); }
__device__ __forceinline__ void fma4(float4& acc, float s, const float4& v) {
  acc.x = fmaf(s, v.x, acc.x);
  acc.y = fmaf(s, v.y, acc.y);
  acc.z = fmaf(s, v.z, acc.z);
  acc.w = fmaf(s, v.w, acc.w);
}

// 4 consecutive stored values <-> float4 (storage types of the precision form:
// float, bfloat16, half; uint16 counts).  Conversions to storage round to
// nearest.  A bfloat16 is the upper half of the float32 with the same value,
// so widening is one shift or mask per value (exact); measured at full size
// against the conversion intrinsic: forward 1.47 vs 1.60 ms, back-projection
// 1.99 vs 2.15 ms.
__device__ __forceinline__ float4 load4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float4 load4(const __nv_bfloat16* p) {
  const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
  return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                     __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
}
__device__ __forceinline__ float4 load4(const __half* p) {
  const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
  return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float4 load4(const uint16_t* p) {
  const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
  return make_float4((float)(u.x & 0xffffu), (float)(u.x >> 16), (float)(u.y & 0xffffu),
                     (float)(u.y >> 16));
}
// plain (non-__ldg) loads for in-place read-modify-write of the image
__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float4 ld4(const __nv_bfloat16* p) {
  const uint2 u = *reinterpret_cast<const uint2*>(p);
  return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                     __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
}
__device__ __forceinline__ float4 ld4(const __half* p) {
  const uint2 u = *reinterpret_cast<const uint2*>(p);
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
  return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ void st4(__nv_bfloat16* p, float4 v) {
  uint2 u;
  *reinterpret_cast<__nv_bfloat162*>(&u.x) = __float22bfloat162_rn(make_float2(v.x, v.y));
  *reinterpret_cast<__nv_bfloat162*>(&u.y) = __float22bfloat162_rn(make_float2(v.z, v.w));
  *reinterpret_cast<uint2*>(p) = u;
}
__device__ __forceinline__ void st4(__half* p, float4 v) {
  // saturate to the largest finite half instead of overflowing to infinity
  const float mx = 65504.f;
  v = make_float4(fminf(v.x, mx), fminf(v.y, mx), fminf(v.z, mx), fminf(v.w, mx));
  uint2 u;
  *reinterpret_cast<__half2*>(&u.x) = __float22half2_rn(make_float2(v.x, v.y));
  *reinterpret_cast<__half2*>(&u.y) = __float22half2_rn(make_float2(v.z, v.w));
  *reinterpret_cast<uint2*>(p) = u;
}
__device__ __forceinline__ float4 mul4(float4 a, float4 b) {
  return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w);
}

// Fractional minor index of centred bin bf given inner = fma(tf, gamma, centre)
// (shared by both kernels, explicit fused multiply-adds: identical bits).
__device__ __forceinline__ float minor_pos(float bf, float beta, float inner) {
  return __fmaf_rn(bf, beta, inner);
}
__device__ __forceinline__ float inner_pos(float tf, float gamma, float centre) {
  return __fmaf_rn(tf, gamma, centre);
}

struct ProjArgs {
  const void* x;          // image (forward input / OSL in-out), storage type TX
  void* xout;             // image output (back-projection)
  const void* y;          // subset sinogram input (back-projection), storage type TY
  void* yout;             // subset sinogram output (forward)
  int yq;                 // 4-frame quads per bin row of y / yout (MQ: dense rows)
  const float4* xscale;   // per-frame scale of a stored image [MQ] (null: 1)
  const AngleTab* ang;
  const int* sub;         // angle indices of the subset
  int n_sub;
  int nx, ny, nz, B, A;
  // ratio / OSL terms
  const void* counts;     // [Z][A][B][M], storage type TC
  const float4* randoms;  // per frame [MQ] or full [Z][A][B][MQ]
  int randoms_layout;
  const float* bin_factor;  // [Z][A][B] or null
  const float4* dt;         // [MQ]
  float kappa;
  const float4* F;          // model TACs or null
  float prior_scale;        // beta / (S sigma2)
  double* ll_partial;       // non-null: accumulate the log-likelihood, no ratio
  int pair_all;             // every angle obeys the pair rule (AngleTab::pair)
  const float4* yscale;     // per-frame scale of a stored sinogram (back-projection input) or null
  int aligned32;            // x, xout and F start on 32-byte boundaries
  float max_beta, max_gamma;   // largest |beta| and |gamma| over the launch's angles
};

constexpr int LL_PARTS = 1024;   // partial sums of the log-likelihood

// Conservative major-step range [t0, t1] where the ray of centred bin bf can
// touch the grid; the exact in-grid test is made per step.
__device__ __forceinline__ void ray_range(float bf, const AngleTab& T, int n_major, int n_minor,
                                          float centre, float tc, int& t0, int& t1) {
  t0 = 0;
  t1 = n_major - 1;
  const float base = __fmaf_rn(bf, T.beta, centre);
  if (fabsf(T.gamma) > 1e-6f) {
    const float ta = (-1.0f - base) / T.gamma + tc;
    const float tb = ((float)n_minor - base) / T.gamma + tc;
    const float lo = fminf(ta, tb), hi = fmaxf(ta, tb);
    t0 = max(0, (int)floorf(fmaxf(lo, -4.0f)) - 2);
    t1 = min(n_major - 1, (int)ceilf(fminf(hi, (float)n_major + 4.0f)) + 2);
  }
}

// Epilogue of ray (z, ak, b) for this lane's frame quad q: the weighted sum
// as the projection, or with RATIO the ratio s / (kappa dt n_d (P x) + r) (or,
// with ll_partial, the Poisson log-likelihood terms instead of the ratio).
template <int MQ, bool RATIO, class TC, class TY>
__device__ __forceinline__ void fwd_epilogue(const ProjArgs& p, float4 acc, float w, int z, int ak,
                                             int a, int b, int q) {
  acc.x *= w; acc.y *= w; acc.z *= w; acc.w *= w;
  if (p.xscale) acc = mul4(acc, __ldg(p.xscale + q));     // stored image -> activity
  const size_t oi = ((size_t)(z * p.n_sub + ak) * p.B + b) * p.yq + q;
  if (!RATIO) {
    st4(static_cast<TY*>(p.yout) + oi * 4, acc);
    return;
  }
  const size_t bin = (size_t)(z * p.A + a) * p.B + b;
  const float nd = p.bin_factor ? __ldg(p.bin_factor + bin) : 1.0f;
  const float4 dt = __ldg(p.dt + q);
  const float4 s = load4(static_cast<const TC*>(p.counts) + (bin * MQ + q) * 4);
  float4 r = f4(0.f);
  if (p.randoms_layout == KCS_RANDOMS_PER_FRAME) r = __ldg(p.randoms + q);
  else if (p.randoms_layout == KCS_RANDOMS_FULL) r = __ldg(p.randoms + bin * MQ + q);
  const float kn = p.kappa * nd;
  float4 yb, rho;
  yb.x = fmaf(kn * dt.x, acc.x, r.x);
  yb.y = fmaf(kn * dt.y, acc.y, r.y);
  yb.z = fmaf(kn * dt.z, acc.z, r.z);
  yb.w = fmaf(kn * dt.w, acc.w, r.w);
  if (p.ll_partial) {
    // Poisson log-likelihood terms s log ybar - ybar of this lane's 4 frames
    // (log s! dropped; s log ybar taken as 0 where ybar <= 0)
    const float t = (yb.x > 0.f ? s.x * logf(yb.x) : 0.f) - yb.x +
                    (yb.y > 0.f ? s.y * logf(yb.y) : 0.f) - yb.y +
                    (yb.z > 0.f ? s.z * logf(yb.z) : 0.f) - yb.z +
                    (yb.w > 0.f ? s.w * logf(yb.w) : 0.f) - yb.w;
    atomicAdd(p.ll_partial + (blockIdx.x & (LL_PARTS - 1)), (double)t);
    return;
  }
  rho.x = yb.x > 0.f ? __fdividef(s.x, yb.x) : 0.f;
  rho.y = yb.y > 0.f ? __fdividef(s.y, yb.y) : 0.f;
  rho.z = yb.z > 0.f ? __fdividef(s.z, yb.z) : 0.f;
  rho.w = yb.w > 0.f ? __fdividef(s.w, yb.w) : 0.f;
  st4(static_cast<TY*>(p.yout) + oi * 4, rho);
}

// Forward projection of every frame of rays (z, ak, b); RATIO replaces the
// projection by rho = s / (kappa dt n_d (P x) + r).
constexpr int FWD_THREADS = 128;   // 4 warps per block (measured best of 64..512)
// Register budget and steps per trip of the march, by image storage type.
// Float32: 8 blocks per SM, a 64-register budget that keeps 8 steps' loads
// in flight (1.50 ms per subset at full size, against 1.68 ms with the
// default budget of 40 registers and 4 steps; 6-10 blocks and 4-12 steps
// measured 1.50-1.56 ms).  16-bit storage: the widening needs registers of
// its own; the default budget (63 registers) with 4 steps is best (bf16
// 1.47 ms; 6 or 8 steps at 78-96 registers 1.58-1.63 ms, 8 steps at 64
// registers spilled 180 bytes and took 3.3 ms).
#ifndef KCS_FWD16_MIN_BLOCKS
#define KCS_FWD16_MIN_BLOCKS 1
#endif
#ifndef KCS_FWD16_STEPS
#define KCS_FWD16_STEPS 4
#endif
template <class TX> struct FwdTune {
  static constexpr int min_blocks = 8, steps = 8;
};
template <> struct FwdTune<__nv_bfloat16> {
  static constexpr int min_blocks = KCS_FWD16_MIN_BLOCKS, steps = KCS_FWD16_STEPS;
};
template <> struct FwdTune<__half> {
  static constexpr int min_blocks = KCS_FWD16_MIN_BLOCKS, steps = KCS_FWD16_STEPS;
};

template <int MQ, bool RATIO, class TX, class TC, class TY>
__global__ void __launch_bounds__(FWD_THREADS, FwdTune<TX>::min_blocks) k_forward(ProjArgs p) {
  constexpr int RPW = 32 / MQ;
  const int lane = threadIdx.x & 31;
  const int sub = lane / MQ;
  const int q = lane - sub * MQ;
  if (sub >= RPW) return;
  const long long ray = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * RPW + sub;
  const long long n_rays = (long long)p.nz * p.n_sub * p.B;
  if (ray >= n_rays) return;
  const int b = (int)(ray % p.B);
  const long long zr = ray / p.B;
  const int ak = (int)(zr % p.n_sub);
  const int z = (int)(zr / p.n_sub);
  const int a = p.sub[ak];
  const AngleTab T = p.ang[a];
  const int n_major = T.xmajor ? p.nx : p.ny;
  const int n_minor = T.xmajor ? p.ny : p.nx;
  const int s_major = T.xmajor ? 4 * MQ : p.nx * 4 * MQ;   // element stride of a major step
  const int s_minor = T.xmajor ? p.nx * 4 * MQ : 4 * MQ;   // element stride of a minor step
  const float tc = 0.5f * (float)(n_major - 1);
  const float centre = 0.5f * (float)(n_minor - 1);
  const float bf = (float)b - 0.5f * (float)(p.B - 1);
  const TX* xz = static_cast<const TX*>(p.x) + ((size_t)z * p.ny * p.nx * MQ + q) * 4;

  // Conservative major-step range where the ray can touch the grid; the exact
  // test is repeated per step below.
  int t0, t1;
  ray_range(bf, T, n_major, n_minor, centre, tc, t0, t1);
  // Branch-free march, U steps per trip: out-of-grid partners are predicated
  // loads of zero (their weight is exactly 0), so several steps' loads are in
  // flight at once and the accumulated values equal the plain loop's.
  float4 acc = f4(0.f);
  constexpr int U = FwdTune<TX>::steps;
  const unsigned nmin = (unsigned)n_minor;
  // per trip: the centred major coordinate of its first step (exact: small
  // integers and half-integers) and the image row/column of that step; within
  // a trip the offsets are 32-bit (a plane holds fewer than 2^31 elements)
  float tf = (float)t0 - tc;
  const TX* xt = xz + (ptrdiff_t)t0 * s_major;
  for (int tb = t0; tb <= t1; tb += U, tf += (float)U, xt += (ptrdiff_t)U * s_major) {
    float4 v0[U], v1[U];
    float w0[U], w1[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool live = tb + u <= t1;
      const float fr = minor_pos(bf, T.beta, inner_pos(tf + (float)u, T.gamma, centre));
      const float fl = floorf(fr);
      const int j0 = (int)fl;
      const float f = fr - fl;
      const bool in0 = live && (unsigned)j0 < nmin;
      const bool in1 = live && (unsigned)(j0 + 1) < nmin;
      const TX* px = xt + (u * s_major + j0 * s_minor);
      v0[u] = in0 ? load4(px) : f4(0.f);
      v1[u] = in1 ? load4(px + s_minor) : f4(0.f);
      w0[u] = in0 ? 1.0f - f : 0.f;
      w1[u] = in1 ? f : 0.f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      fma4(acc, w0[u], v0[u]);
      fma4(acc, w1[u], v1[u]);
    }
  }
  fwd_epilogue<MQ, RATIO, TC, TY>(p, acc, T.w, z, ak, a, b, q);
}

__device__ __forceinline__ void ld8(const float* p, float4& a, float4& b) {   // read-only
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
      : "l"(p));
}
__device__ __forceinline__ void ld8c(const float* p, float4& a, float4& b) {   // coherent
  asm volatile("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z),
                 "=f"(b.w)
               : "l"(p));
}
__device__ __forceinline__ void st8(float* p, const float4& a, const float4& b) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(a.x),
               "f"(a.y), "f"(a.z), "f"(a.w), "f"(b.x), "f"(b.y), "f"(b.z), "f"(b.w)
               : "memory");
}
// The OSL update of one frame quad (Eq. 2-3): x <- x kappa dt acc / den.
__device__ __forceinline__ float4 osl_quad(float4 xv, const float4* Fv, float4 dt, float ks,
                                          float ps, float kappa, float4 acc) {
  float4 den = make_float4(dt.x * ks, dt.y * ks, dt.z * ks, dt.w * ks);
  if (Fv) {
    den.x = fmaxf(fmaf(ps, xv.x - Fv->x, den.x), 1e-3f * den.x);
    den.y = fmaxf(fmaf(ps, xv.y - Fv->y, den.y), 1e-3f * den.y);
    den.z = fmaxf(fmaf(ps, xv.z - Fv->z, den.z), 1e-3f * den.z);
    den.w = fmaxf(fmaf(ps, xv.w - Fv->w, den.w), 1e-3f * den.w);
  }
  xv.x = __fdividef(xv.x * (kappa * dt.x * acc.x), den.x);
  xv.y = __fdividef(xv.y * (kappa * dt.y * acc.y), den.y);
  xv.z = __fdividef(xv.z * (kappa * dt.z * acc.z), den.z);
  xv.w = __fdividef(xv.w * (kappa * dt.w * acc.w), den.w);
  return xv;
}

__global__ void k_sum_parts(const double* parts, int n, double* out) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += parts[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// Bins whose sample at this major step can land in [m-1, m+1): the real-valued
// position b*beta + inner differs from the kernels' single fused multiply-add by
// half an ulp (< 1e-4 of a step at these sizes), so a 1e-3 margin on the
// real-valued bin interval is conservative; the exact test is made per
// candidate by the caller.
__device__ __forceinline__ void bin_range_tight(const AngleTab& T, int m, float inner, float bc,
                                                int B, int& b_lo, int& b_hi) {
  float lo = ((float)(m - 1) - inner) * T.inv_beta;
  float hi = ((float)(m + 1) - inner) * T.inv_beta;
  if (lo > hi) { const float tmp = lo; lo = hi; hi = tmp; }
  b_lo = max(0, (int)ceilf(fmaxf(lo + bc - 1e-3f, -2.0f)));
  b_hi = min(B - 1, (int)floorf(fminf(hi + bc + 1e-3f, (float)B + 2.0f)));
}

// Bins of angle T whose sample at major step t lands within one minor step of
// m, with one extra bin of margin on each side (used to bound staged tiles):
// the exact test is made per candidate by the caller.
__device__ __forceinline__ void bin_range(const AngleTab& T, int m, float inner, float bc, int B,
                                          int& b_lo, int& b_hi) {
  float lo = ((float)(m - 1) - inner) * T.inv_beta;
  float hi = ((float)(m + 1) - inner) * T.inv_beta;
  if (lo > hi) { const float tmp = lo; lo = hi; hi = tmp; }
  b_lo = max(0, (int)floorf(fmaxf(lo + bc, -2.0f)) - 1);
  b_hi = min(B - 1, (int)ceilf(fminf(hi + bc, (float)B + 2.0f)) + 1);
}

// Tiled gather back-projection: one thread per voxel of a 16 x 16 in-plane
// tile, all frames per thread (the candidate-bin geometry is computed once per
// voxel and angle).  The ratio rows the tile can touch are staged in shared
// memory, up to BK_ACHUNK angles at a time, with an odd 16-byte row pitch so
// that the per-thread 128-bit reads of different rows fall in different banks.
// MODE 0: x = P_k^T y.  MODE 1: OSL update of x in place with y = rho.
constexpr int BK_TILE = 16;
constexpr int BK_ACHUNK = 12;

__host__ __device__ constexpr int bk_pitch(int MQ) { return MQ | 1; }

template <int MQ, int MODE, class TX, class TY>
__global__ void __launch_bounds__(BK_TILE * BK_TILE) k_back_tiled(ProjArgs p, int rows_max,
                                                                   int achunk) {
  constexpr int PITCH = bk_pitch(MQ);
  extern __shared__ float4 srho[];           // [achunk][rows_max][PITCH]
  __shared__ int s_lo[BK_ACHUNK], s_cnt[BK_ACHUNK], s_a[BK_ACHUNK];
  __shared__ AngleTab s_T[BK_ACHUNK];
  const int ntx = (p.nx + BK_TILE - 1) / BK_TILE;
  const int nty = (p.ny + BK_TILE - 1) / BK_TILE;
  const int tile = blockIdx.x;
  const int tx = tile % ntx;
  const int ty = (tile / ntx) % nty;
  const int z = tile / (ntx * nty);
  const int i0 = tx * BK_TILE, j0 = ty * BK_TILE;
  const int i1 = min(i0 + BK_TILE, p.nx) - 1, j1 = min(j0 + BK_TILE, p.ny) - 1;
  const int i = i0 + (threadIdx.x % BK_TILE);
  const int j = j0 + (threadIdx.x / BK_TILE);
  const bool valid = i < p.nx && j < p.ny;
  const float bc = 0.5f * (float)(p.B - 1);
  float4 acc[MQ];
#pragma unroll
  for (int q = 0; q < MQ; ++q) acc[q] = f4(0.f);
  float sens = 0.f;
  for (int a0 = 0; a0 < p.n_sub; a0 += achunk) {
    const int na = min(achunk, p.n_sub - a0);
    if ((int)threadIdx.x < na) {
      // union of the candidate ranges of the tile's four corners
      const int a = p.sub[a0 + threadIdx.x];
      const AngleTab T = p.ang[a];
      s_a[threadIdx.x] = a;
      s_T[threadIdx.x] = T;
      const int n_major = T.xmajor ? p.nx : p.ny;
      const int n_minor = T.xmajor ? p.ny : p.nx;
      const float tc = 0.5f * (float)(n_major - 1);
      const float centre = 0.5f * (float)(n_minor - 1);
      const int ta = T.xmajor ? i0 : j0, tb = T.xmajor ? i1 : j1;
      const int ma = T.xmajor ? j0 : i0, mb = T.xmajor ? j1 : i1;
      int lo = p.B, hi = -1;
      for (int c = 0; c < 4; ++c) {
        const int t = (c & 1) ? tb : ta;
        const int m = (c & 2) ? mb : ma;
        int l, h;
        bin_range(T, m, inner_pos((float)t - tc, T.gamma, centre), bc, p.B, l, h);
        lo = min(lo, l);
        hi = max(hi, h);
      }
      lo = max(0, lo - 1);
      hi = min(p.B - 1, hi + 1);
      s_lo[threadIdx.x] = lo;
      s_cnt[threadIdx.x] = max(0, min(hi - lo + 1, rows_max));
    }
    __syncthreads();
    for (int c = 0; c < na; ++c) {
      const TY* src = static_cast<const TY*>(p.y) +
                      ((size_t)(z * p.n_sub + a0 + c) * p.B + s_lo[c]) * p.yq * 4;
      float4* dst = srho + (size_t)c * rows_max * PITCH;
      const int n = s_cnt[c] * MQ;
      for (int e = threadIdx.x; e < n; e += BK_TILE * BK_TILE) {
        const int r = e / MQ, q = e - r * MQ;
        dst[r * PITCH + q] = load4(src + ((size_t)r * p.yq + q) * 4);
      }
    }
    __syncthreads();
    if (valid) {
      for (int c = 0; c < na; ++c) {
        const int a = s_a[c];
        const AngleTab T = s_T[c];
        const int n_major = T.xmajor ? p.nx : p.ny;
        const int n_minor = T.xmajor ? p.ny : p.nx;
        const int t = T.xmajor ? i : j;
        const int m = T.xmajor ? j : i;
        const float tc = 0.5f * (float)(n_major - 1);
        const float centre = 0.5f * (float)(n_minor - 1);
        const float inner = inner_pos((float)t - tc, T.gamma, centre);
        int b_lo, b_hi;
        bin_range_tight(T, m, inner, bc, p.B, b_lo, b_hi);
        const int lo = s_lo[c];
        b_lo = max(b_lo, lo);
        b_hi = min(b_hi, lo + s_cnt[c] - 1);
        const float4* rows = srho + (size_t)c * rows_max * PITCH;
        const size_t binrow = (size_t)(z * p.A + a) * p.B;
        for (int b = b_lo; b <= b_hi; ++b) {
          const float fr = minor_pos((float)b - bc, T.beta, inner);
          const float fl = floorf(fr);
          const int jj = (int)fl;
          const float f = fr - fl;
          float wt = (jj == m) ? 1.0f - f : ((jj + 1 == m) ? f : 0.0f);
          if (wt == 0.0f) continue;
          wt *= T.w;
          if (MODE == 1 && p.bin_factor) wt *= __ldg(p.bin_factor + binrow + b);
          const float4* row = rows + (b - lo) * PITCH;
#pragma unroll
          for (int q = 0; q < MQ; ++q) fma4(acc[q], wt, row[q]);
          sens += wt;
        }
      }
    }
    __syncthreads();
  }
  if (!valid) return;
  const size_t vi = ((size_t)(z * p.ny + j) * p.nx + i) * MQ;
  if (MODE == 0) {
#pragma unroll
    for (int q = 0; q < MQ; ++q)
      st4(static_cast<TX*>(p.xout) + (vi + q) * 4,
          p.yscale ? mul4(acc[q], __ldg(p.yscale + q)) : acc[q]);   // stored sinogram -> value
    return;
  }
  if (!(sens > 0.f)) return;   // x unchanged where no ray of the subset sees the voxel
  const float ks = p.kappa * sens;
#pragma unroll
  for (int q = 0; q < MQ; ++q) {
    float4 xv = ld4(static_cast<const TX*>(p.x) + (vi + q) * 4);
    const float4 sc = p.xscale ? __ldg(p.xscale + q) : f4(1.f);
    if (p.xscale) xv = mul4(xv, sc);            // stored image -> activity
    const float4 dt = __ldg(p.dt + q);
    float4 den = make_float4(dt.x * ks, dt.y * ks, dt.z * ks, dt.w * ks);
    if (p.F) {
      const float4 Fv = __ldg(p.F + vi + q);
      const float ps = p.prior_scale;
      den.x = fmaxf(fmaf(ps, xv.x - Fv.x, den.x), 1e-3f * den.x);
      den.y = fmaxf(fmaf(ps, xv.y - Fv.y, den.y), 1e-3f * den.y);
      den.z = fmaxf(fmaf(ps, xv.z - Fv.z, den.z), 1e-3f * den.z);
      den.w = fmaxf(fmaf(ps, xv.w - Fv.w, den.w), 1e-3f * den.w);
    }
    // a stored 16-bit image: activity -> stored value in the one division
    if (!std::is_same<TX, float>::value && p.xscale) den = mul4(den, sc);
    xv.x = __fdividef(xv.x * (p.kappa * dt.x * acc[q].x), den.x);
    xv.y = __fdividef(xv.y * (p.kappa * dt.y * acc[q].y), den.y);
    xv.z = __fdividef(xv.z * (p.kappa * dt.z * acc[q].z), den.z);
    xv.w = __fdividef(xv.w * (p.kappa * dt.w * acc[q].w), den.w);
    if (std::is_same<TX, float>::value && p.xscale)
      xv = make_float4(xv.x / sc.x, xv.y / sc.y, xv.z / sc.z, xv.w / sc.w);
    st4(static_cast<TX*>(p.xout) + (vi + q) * 4, xv);
  }
}

// ------------------------------------------------------------ bulk-copy staging
// Device-side count of bounded waits that ran out (a broken invariant, never
// expected); read by kcs_device_status.
__device__ unsigned int g_wait_timeouts;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
// Arrive on bar (count 1) announcing `bytes` of asynchronous copies.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// One bulk copy global -> this CTA's shared memory, completion counted on bar.
// dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for phase `parity` of bar; false (and the device counter
// raised) if it did not complete within the limit.
constexpr int MBAR_SPIN_LIMIT = 1 << 22;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (int it = 0; it < MBAR_SPIN_LIMIT; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  atomicAdd(&g_wait_timeouts, 1u);
  return false;
}

// Failure-detection self-test: a barrier nothing arrives on, waited for with a
// small limit; the wait runs out and raises the counter like a real timeout.
__global__ void k_selftest_wait(int limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  bool done = false;
  for (int it = 0; it < limit && !done; ++it) done = mbar_try_wait(&bar, 0);
  if (!done && threadIdx.x == 0) atomicAdd(&g_wait_timeouts, 1u);
}

// Forward projection with the image staged in shared memory.  A block takes
// SF_RAYS consecutive bins of one plane and angle and marches them together in
// chunks of SF_T major steps.  For each chunk, warp 0 bulk-copies the window
// of the plane those rays can touch (the rows or columns of the chunk, over
// `span` minor positions around the rays) into one of two shared buffers while
// the block works on the other; the interpolation partners are then read from
// shared memory.  Each ray sums its samples in the same order as k_forward
// (steps ascending, left then right partner), so both kernels give the same
// bits.  Layouts: y-major angles [SF_T][span][M] (a staged row is a piece of
// one image row); x-major angles [span][xpitch] with SF_T voxels of one image
// row each and xpitch = M (mod 32) floats, so that neighbouring rays' partners
// fall in different banks.  Window positions outside the grid, and buffer
// parts no copy filled, hold finite values that only zero weights meet.
constexpr int SF_WARPS = 4;
constexpr int SF_T = 4;

struct StagedDims {
  int span;     // minor positions per chunk window
  int xpitch;   // floats per staged row of an x-major window
  int buf;      // floats per buffer
};

template <int MQ>
__device__ __forceinline__ int staged_window(const AngleTab& T, float bf0, float bf1, int t0,
                                             float tc, float centre) {
  // lowest minor index any partner of the chunk can have, less a margin of one
  const float i0 = inner_pos((float)t0 - tc, T.gamma, centre);
  const float i1 = inner_pos((float)(t0 + SF_T - 1) - tc, T.gamma, centre);
  const float m = fminf(fminf(minor_pos(bf0, T.beta, i0), minor_pos(bf1, T.beta, i0)),
                        fminf(minor_pos(bf0, T.beta, i1), minor_pos(bf1, T.beta, i1)));
  return (int)floorf(m) - 1;
}

template <int MQ, bool RATIO, class TC, class TY>
__global__ void __launch_bounds__(SF_WARPS * 32) k_forward_staged(ProjArgs p, StagedDims d) {
  constexpr int RPW = 32 / MQ;
  constexpr int R = SF_WARPS * RPW;   // rays per block
  constexpr int M = 4 * MQ;
  extern __shared__ __align__(16) float sbuf[];   // [2][d.buf]
  __shared__ __align__(8) uint64_t s_bar[2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sub = lane / MQ;
  const int q = lane - sub * MQ;
  const int gpr = (p.B + R - 1) / R;
  const int gb = (int)(blockIdx.x % gpr);
  const int zr = (int)(blockIdx.x / gpr);
  const int ak = zr % p.n_sub;
  const int z = zr / p.n_sub;
  const int a = p.sub[ak];
  const AngleTab T = p.ang[a];
  const int n_major = T.xmajor ? p.nx : p.ny;
  const int n_minor = T.xmajor ? p.ny : p.nx;
  const float tc = 0.5f * (float)(n_major - 1);
  const float centre = 0.5f * (float)(n_minor - 1);
  const float bc = 0.5f * (float)(p.B - 1);
  const int b_first = gb * R, b_last = min(p.B, b_first + R) - 1;
  const int b = b_first + warp * RPW + sub;
  const bool ray_on = sub < RPW && b < p.B;
  const float bf = (float)b - bc;
  const float bf0 = (float)b_first - bc, bf1 = (float)b_last - bc;
  // the block's major range: the union of its rays' ranges (monotone in the bin)
  int t_start, t_end;
  {
    int r0, r1, s0, s1;
    ray_range(bf0, T, n_major, n_minor, centre, tc, r0, r1);
    ray_range(bf1, T, n_major, n_minor, centre, tc, s0, s1);
    t_start = min(r0, s0);
    t_end = max(r1, s1);
  }
  const int nch = t_end >= t_start ? (t_end - t_start) / SF_T + 1 : 0;
  const float* xz = static_cast<const float*>(p.x) + (size_t)z * p.ny * p.nx * M;
  for (int i = threadIdx.x; i < 2 * d.buf; i += SF_WARPS * 32) sbuf[i] = 0.f;
  if (threadIdx.x == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // warp 0: copy chunk c's window into buffer `buf`
  auto issue = [&](int c, int buf) {
    const int t0 = t_start + c * SF_T;
    const int jlo = staged_window<MQ>(T, bf0, bf1, t0, tc, centre);
    float* dst0 = sbuf + (size_t)buf * d.buf;
    const int rows = T.xmajor ? d.span : SF_T;
    uint32_t bytes = 0;
    for (int r = lane; r < rows; r += 32) {
      int len;
      if (T.xmajor) {
        const int j = jlo + r;
        len = (j >= 0 && j < n_minor) ? min(SF_T, n_major - t0) : 0;
      } else {
        const int t = t0 + r;
        len = t < n_major ? min(jlo + d.span, n_minor) - max(jlo, 0) : 0;
      }
      bytes += (uint32_t)max(len, 0) * M * 4;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
    // earlier generic accesses of the buffer (ordered by the block barrier)
    // before the asynchronous copies that overwrite it
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (lane == 0) mbar_expect_tx(&s_bar[buf], bytes);
    __syncwarp();
    for (int r = lane; r < rows; r += 32) {
      const float* src;
      float* dst;
      int len;
      if (T.xmajor) {   // minor = y = jlo + r, major = x in [t0, t0 + SF_T)
        const int j = jlo + r;
        len = (j >= 0 && j < n_minor) ? min(SF_T, n_major - t0) : 0;
        src = xz + ((size_t)j * p.nx + t0) * M;
        dst = dst0 + (size_t)r * d.xpitch;
      } else {          // major = y = t0 + r, minor = x in [jlo, jlo + span)
        const int t = t0 + r;
        const int c0 = max(jlo, 0);
        len = t < n_major ? min(jlo + d.span, n_minor) - c0 : 0;
        src = xz + ((size_t)t * p.nx + c0) * M;
        dst = dst0 + ((size_t)r * d.span + (c0 - jlo)) * M;
      }
      if (len > 0) bulk_g2s(dst, src, (uint32_t)len * M * 4, &s_bar[buf]);
    }
  };
  if (warp == 0) {
    if (nch > 0) issue(0, 0);
    if (nch > 1) issue(1, 1);
  }
  const unsigned nmin = (unsigned)n_minor;
  const int s_step = T.xmajor ? M : d.span * M;        // floats per major step in a window
  const int s_minor = T.xmajor ? d.xpitch : M;         // floats per minor step in a window
  float4 acc = f4(0.f);
  bool ok = true;
  for (int c = 0; c < nch; ++c) {
    const int buf = c & 1;
    ok = mbar_wait(&s_bar[buf], (uint32_t)(c >> 1) & 1u) && ok;
    const int t0 = t_start + c * SF_T;
    const int jlo = staged_window<MQ>(T, bf0, bf1, t0, tc, centre);
    const float* sb = sbuf + (size_t)buf * d.buf + q * 4;
    if (ray_on && ok) {
      float tf = (float)t0 - tc;
#pragma unroll
      for (int u0 = 0; u0 < SF_T; u0 += 4) {
        float4 v0[4], v1[4];
        float w0[4], w1[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int t = t0 + u0 + u;
          const bool live = t <= t_end;
          const float fr = minor_pos(bf, T.beta, inner_pos(tf + (float)(u0 + u), T.gamma, centre));
          const float fl = floorf(fr);
          const int j0 = (int)fl;
          const float f = fr - fl;
          const bool in0 = live && (unsigned)j0 < nmin;
          const bool in1 = live && (unsigned)(j0 + 1) < nmin;
          // in the window by construction (corner extremes); the clamp only
          // keeps every shared-memory read inside the buffer
          const int rel = min(max(j0 - jlo, 0), d.span - 2);
          const float* ps = sb + (u0 + u) * s_step + rel * s_minor;
          v0[u] = in0 ? *reinterpret_cast<const float4*>(ps) : f4(0.f);
          v1[u] = in1 ? *reinterpret_cast<const float4*>(ps + s_minor) : f4(0.f);
          w0[u] = in0 ? 1.0f - f : 0.f;
          w1[u] = in1 ? f : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          fma4(acc, w0[u], v0[u]);
          fma4(acc, w1[u], v1[u]);
        }
      }
    }
    __syncthreads();   // buffer `buf` read by every warp
    if (warp == 0 && c + 2 < nch) issue(c + 2, buf);
  }
  if (!ok) {
    // a wait ran out: wait (bounded) for the copies still in flight
    for (int c = max(0, nch - 2); c < nch; ++c) mbar_wait(&s_bar[c & 1], (uint32_t)(c >> 1) & 1u);
    return;
  }
  if (ray_on) fwd_epilogue<MQ, RATIO, TC, TY>(p, acc, T.w, z, ak, a, b, q);
}

// The tiled gather back-projection of k_back_tiled with the ratio rows of
// each angle brought into shared memory by one bulk copy (the rows of one
// angle and plane are contiguous in the [Z][A_k][B][M] sinogram), issued by a
// single thread for all angles of the chunk at once; every thread waits only
// for the angle it is about to use, so the copies of later angles overlap the
// work on earlier ones and no thread spends issue slots on staging.  Rows are
// dense in shared memory (pitch = one bin's frames).
template <int MQ, int MODE, class TX, class TY, bool PAIR>
__global__ void __launch_bounds__(BK_TILE * BK_TILE, 4) k_back_bulk(ProjArgs p, int rows_max,
                                                                  int achunk) {
  // bytes of one bin row: p.yq quads, a multiple of 16 (checked by the launcher)
  const int RB = p.yq * 4 * (int)sizeof(TY);
  extern __shared__ __align__(16) unsigned char sraw[];   // [achunk][rows_max] rows
  __shared__ int s_lo[BK_ACHUNK], s_cnt[BK_ACHUNK], s_a[BK_ACHUNK];
  __shared__ AngleTab s_T[BK_ACHUNK];
  __shared__ __align__(8) uint64_t s_bar[BK_ACHUNK];
  const int ntx = (p.nx + BK_TILE - 1) / BK_TILE;
  const int nty = (p.ny + BK_TILE - 1) / BK_TILE;
  const int tile = blockIdx.x;
  const int tx = tile % ntx;
  const int ty = (tile / ntx) % nty;
  const int z = tile / (ntx * nty);
  const int i0 = tx * BK_TILE, j0 = ty * BK_TILE;
  const int i1 = min(i0 + BK_TILE, p.nx) - 1, j1 = min(j0 + BK_TILE, p.ny) - 1;
  const int i = i0 + (threadIdx.x % BK_TILE);
  const int j = j0 + (threadIdx.x / BK_TILE);
  const bool valid = i < p.nx && j < p.ny;
  const float bc = 0.5f * (float)(p.B - 1);
  if (threadIdx.x == 0) {
    for (int c = 0; c < BK_ACHUNK; ++c) mbar_init(&s_bar[c], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();   // barriers initialised before anyone waits on them
  float4 acc[MQ];
#pragma unroll
  for (int q = 0; q < MQ; ++q) acc[q] = f4(0.f);
  float sens = 0.f;
  bool ok = true;
  uint32_t parity = 0;
  for (int a0 = 0; a0 < p.n_sub; a0 += achunk, parity ^= 1u) {
    const int na = min(achunk, p.n_sub - a0);
    // Warp 0 sets the chunk up while the other warps go straight to waiting on
    // the per-angle barriers: the angle tables it writes become visible to them
    // through the release of the barrier arrive (after a warp barrier) and the
    // acquire of their wait.
    if (threadIdx.x < 32) {
      if ((int)threadIdx.x < na) {
        // union of the candidate ranges of the tile's four corners
        const int a = p.sub[a0 + threadIdx.x];
        const AngleTab T = p.ang[a];
        s_a[threadIdx.x] = a;
        s_T[threadIdx.x] = T;
        const int n_major = T.xmajor ? p.nx : p.ny;
        const int n_minor = T.xmajor ? p.ny : p.nx;
        const float tc = 0.5f * (float)(n_major - 1);
        const float centre = 0.5f * (float)(n_minor - 1);
        const int ta = T.xmajor ? i0 : j0, tb = T.xmajor ? i1 : j1;
        const int ma = T.xmajor ? j0 : i0, mb = T.xmajor ? j1 : i1;
        int lo = p.B, hi = -1;
        for (int c = 0; c < 4; ++c) {
          const int t = (c & 1) ? tb : ta;
          const int m = (c & 2) ? mb : ma;
          int l, h;
          bin_range(T, m, inner_pos((float)t - tc, T.gamma, centre), bc, p.B, l, h);
          lo = min(lo, l);
          hi = max(hi, h);
        }
        lo = max(0, lo - 1);
        hi = min(p.B - 1, hi + 1);
        s_lo[threadIdx.x] = lo;
        s_cnt[threadIdx.x] = max(0, min(hi - lo + 1, rows_max));
        // the same three integers in the entry's spare words: one 48-byte
        // entry per angle is all the pair path reads
        s_T[threadIdx.x].pad_[0] = lo;
        s_T[threadIdx.x].pad_[1] = max(0, min(hi - lo + 1, rows_max));
        s_T[threadIdx.x].pad_[2] = a;
      }
      __syncwarp();
      if (threadIdx.x == 0) {
        // the previous chunk's rows were read by every thread (generic proxy;
        // block barrier at the end of that chunk) before these async copies
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (int c = 0; c < na; ++c) {
          const uint32_t bytes = (uint32_t)s_cnt[c] * RB;
          mbar_expect_tx(&s_bar[c], bytes);
          if (bytes) {
            const char* src = static_cast<const char*>(p.y) +
                              ((size_t)(z * p.n_sub + a0 + c) * p.B + s_lo[c]) * RB;
            bulk_g2s(sraw + (size_t)c * rows_max * RB, src, bytes, &s_bar[c]);
          }
        }
      }
    }
    for (int c = 0; c < na; ++c) {
      ok = mbar_wait(&s_bar[c], parity) && ok;
      if (!valid || !ok) continue;
      const AngleTab T = s_T[c];
      const int a = (MODE == 1 && PAIR) ? T.pad_[2] : s_a[c];
      const int t = T.xmajor ? i : j;
      const int m = T.xmajor ? j : i;
      const float inner = inner_pos((float)t - T.tc, T.gamma, T.centre);
      // candidates: bins within |1/beta| (+1e-3) of the real bin u whose ray
      // meets minor index m; the exact test below decides
      const float u = fmaf((float)m - inner, T.inv_beta, bc);
      const int lo = (MODE == 1 && PAIR) ? T.pad_[0] : s_lo[c];
      const TY* rows = reinterpret_cast<const TY*>(sraw + (size_t)c * rows_max * RB);
      const size_t binrow = (size_t)(z * p.A + a) * p.B;
      if (MODE == 1 && PAIR) {
        // At most two consecutive bins reach this voxel: the last whose sample
        // lies below m and the first at or above it.  The pair is fixed by
        // one exact test of the forward's own position at the bin nearest
        // the real crossing u, so it holds whatever the rounding of u; both
        // candidates are then processed without a loop or a branch, in
        // ascending bin order as the forward's triples are summed (a zero
        // weight adds exactly nothing: the staged ratios are finite).
        const int cnt = T.pad_[1];
        if (cnt == 0) continue;                            // no staged row reaches the tile
        const float mf = (float)m;
        const float kf = rintf(u);
        const float frk = minor_pos(kf - bc, T.beta, inner);
        const bool below = (frk >= mf) == (T.beta > 0.f);    // pair {k - 1, k}
        const float fro = minor_pos((below ? kf - 1.f : kf + 1.f) - bc, T.beta, inner);
        const int b0 = (int)kf - (below ? 1 : 0);
        float frs[2] = {below ? fro : frk, below ? frk : fro};
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int r = b0 + e - lo;                     // staged row of the candidate
          const float fr = frs[e];
          const float fl = floorf(fr);
          const int jj = (int)fl;
          const float f = fr - fl;
          float wt = (jj == m) ? 1.0f - f : ((jj + 1 == m) ? f : 0.0f);
          wt = ((unsigned)r < (unsigned)cnt) ? wt * T.w : 0.0f;
          if (p.bin_factor && wt != 0.0f) wt *= __ldg(p.bin_factor + binrow + b0 + e);
          const TY* row = rows + (size_t)min(max(r, 0), cnt - 1) * p.yq * 4;
#pragma unroll
          for (int q = 0; q < MQ; ++q) fma4(acc[q], wt, ld4(row + q * 4));
          sens += wt;
        }
        continue;
      }
      const int b_lo = max((int)ceilf(u - T.rband), lo);
      const int b_hi = min((int)floorf(u + T.rband), lo + s_cnt[c] - 1);
      for (int b = b_lo; b <= b_hi; ++b) {
        const float fr = minor_pos((float)b - bc, T.beta, inner);
        const float fl = floorf(fr);
        const int jj = (int)fl;
        const float f = fr - fl;
        float wt = (jj == m) ? 1.0f - f : ((jj + 1 == m) ? f : 0.0f);
        // MODE 1 does not branch around zero weights (fewer divergent
        // branches): its staged ratios are finite (s / ybar or 0), so a zero
        // weight adds exactly nothing.  A caller's sinogram (MODE 0) may not be.
        if (MODE == 0 && wt == 0.0f) continue;
        wt *= T.w;
        if (MODE == 1 && p.bin_factor && wt != 0.0f) wt *= __ldg(p.bin_factor + binrow + b);
        const TY* row = rows + (size_t)(b - lo) * p.yq * 4;
#pragma unroll
        for (int q = 0; q < MQ; ++q) fma4(acc[q], wt, ld4(row + q * 4));
        sens += wt;
      }
    }
    if (!ok) {
      // a wait ran out: before this CTA's shared memory can be reused, wait
      // once more (bounded) for every copy of the chunk still in flight
      for (int c = 0; c < na; ++c) mbar_wait(&s_bar[c], parity);
    }
    if (a0 + achunk < p.n_sub) __syncthreads();   // rows are reused by the next chunk
  }
  if (!valid || !ok) return;
  const size_t vi = ((size_t)(z * p.ny + j) * p.nx + i) * MQ;
  if (MODE == 0) {
#pragma unroll
    for (int q = 0; q < MQ; ++q)
      st4(static_cast<TX*>(p.xout) + (vi + q) * 4,
          p.yscale ? mul4(acc[q], __ldg(p.yscale + q)) : acc[q]);   // stored sinogram -> value
    return;
  }
  if (!(sens > 0.f)) return;   // x unchanged where no ray of the subset sees the voxel
  const float ks = p.kappa * sens;
  if constexpr (std::is_same<TX, float>::value && MQ % 2 == 0) {
    if (p.aligned32 && !p.xscale) {
      // image and model frame vectors by 256-bit loads and stores (half the
      // requests of 16-byte ones)
#pragma unroll
      for (int h = 0; h < MQ / 2; ++h) {
        float4 xa, xb, Fa, Fb;
        ld8c(static_cast<const float*>(p.x) + (vi + 2 * h) * 4, xa, xb);
        if (p.F) ld8(reinterpret_cast<const float*>(p.F + vi + 2 * h), Fa, Fb);
        xa = osl_quad(xa, p.F ? &Fa : nullptr, __ldg(p.dt + 2 * h), ks, p.prior_scale, p.kappa,
                      acc[2 * h]);
        xb = osl_quad(xb, p.F ? &Fb : nullptr, __ldg(p.dt + 2 * h + 1), ks, p.prior_scale,
                      p.kappa, acc[2 * h + 1]);
        st8(static_cast<float*>(p.xout) + (vi + 2 * h) * 4, xa, xb);
      }
      return;
    }
  }
#pragma unroll
  for (int q = 0; q < MQ; ++q) {
    float4 xv = ld4(static_cast<const TX*>(p.x) + (vi + q) * 4);
    const float4 sc = p.xscale ? __ldg(p.xscale + q) : f4(1.f);
    if (p.xscale) xv = mul4(xv, sc);            // stored image -> activity
    const float4 dt = __ldg(p.dt + q);
    float4 den = make_float4(dt.x * ks, dt.y * ks, dt.z * ks, dt.w * ks);
    if (p.F) {
      const float4 Fv = __ldg(p.F + vi + q);
      const float ps = p.prior_scale;
      den.x = fmaxf(fmaf(ps, xv.x - Fv.x, den.x), 1e-3f * den.x);
      den.y = fmaxf(fmaf(ps, xv.y - Fv.y, den.y), 1e-3f * den.y);
      den.z = fmaxf(fmaf(ps, xv.z - Fv.z, den.z), 1e-3f * den.z);
      den.w = fmaxf(fmaf(ps, xv.w - Fv.w, den.w), 1e-3f * den.w);
    }
    // a stored 16-bit image: activity -> stored value in the one division
    if (!std::is_same<TX, float>::value && p.xscale) den = mul4(den, sc);
    xv.x = __fdividef(xv.x * (p.kappa * dt.x * acc[q].x), den.x);
    xv.y = __fdividef(xv.y * (p.kappa * dt.y * acc[q].y), den.y);
    xv.z = __fdividef(xv.z * (p.kappa * dt.z * acc[q].z), den.z);
    xv.w = __fdividef(xv.w * (p.kappa * dt.w * acc[q].w), den.w);
    if (std::is_same<TX, float>::value && p.xscale)
      xv = make_float4(xv.x / sc.x, xv.y / sc.y, xv.z / sc.z, xv.w / sc.w);
    st4(static_cast<TX*>(p.xout) + (vi + q) * 4, xv);
  }
}

// Sensitivity sum_{d in S_k} n_d p_vd: the same gather with unit data.
__global__ void __launch_bounds__(256) k_sens(ProjArgs p, float* sens_out) {
  const long long vox = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n_vox = (long long)p.nz * p.ny * p.nx;
  if (vox >= n_vox) return;
  const int i = (int)(vox % p.nx);
  const long long zj = vox / p.nx;
  const int j = (int)(zj % p.ny);
  const int z = (int)(zj / p.ny);
  const float bc = 0.5f * (float)(p.B - 1);
  float sens = 0.f;
  for (int ak = 0; ak < p.n_sub; ++ak) {
    const int a = p.sub[ak];
    const AngleTab T = p.ang[a];
    const int n_major = T.xmajor ? p.nx : p.ny;
    const int n_minor = T.xmajor ? p.ny : p.nx;
    const int t = T.xmajor ? i : j;
    const int m = T.xmajor ? j : i;
    const float tc = 0.5f * (float)(n_major - 1);
    const float centre = 0.5f * (float)(n_minor - 1);
    const float inner = inner_pos((float)t - tc, T.gamma, centre);
    int b_lo, b_hi;
    bin_range_tight(T, m, inner, bc, p.B, b_lo, b_hi);
    const size_t binrow = (size_t)(z * p.A + a) * p.B;
    for (int b = b_lo; b <= b_hi; ++b) {
      const float fr = minor_pos((float)b - bc, T.beta, inner);
      const float fl = floorf(fr);
      const int j0 = (int)fl;
      const float f = fr - fl;
      float wt = (j0 == m) ? 1.0f - f : ((j0 + 1 == m) ? f : 0.0f);
      if (wt == 0.0f) continue;
      wt *= T.w;
      if (p.bin_factor) wt *= __ldg(p.bin_factor + binrow + b);
      sens += wt;
    }
  }
  sens_out[vox] = sens;
}

// ------------------------------------------------------------ reductions
// Deterministic two-pass sums for the start image: per-frame totals of
// counts - randoms, and the total of n_d (P 1)_d = sum_v sens_v.
constexpr int RED_BLOCKS = 512;


template <class T>
__global__ void __launch_bounds__(256) k_partial_sums(const T* data, long long n_rows, int M,
                                                      double* partial /*[RED_BLOCKS][M]*/) {
  __shared__ double sh[256];
  const int tid = threadIdx.x;
  const long long per = (n_rows + gridDim.x - 1) / gridDim.x;
  const long long r0 = (long long)blockIdx.x * per;
  const long long r1 = min(n_rows, r0 + per);
  for (int m = 0; m < M; ++m) {
    double s = 0.0;
    for (long long r = r0 + tid; r < r1; r += blockDim.x) s += (double)ld1(data + r * M + m);
    sh[tid] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (tid < w) sh[tid] += sh[tid + w];
      __syncthreads();
    }
    if (tid == 0) partial[(size_t)blockIdx.x * M + m] = sh[0];
    __syncthreads();
  }
}

__global__ void k_init_fill(const double* pc, const double* pr, const double* ps,
                            int rand_per_frame, const float* rpf, long long n_bins_total,
                            const float* dt, float kappa, int M, float* cval) {
  const int m = threadIdx.x;
  if (m >= M) return;
  double sc = 0.0, sr = 0.0, ss = 0.0;
  for (int b = 0; b < RED_BLOCKS; ++b) {
    sc += pc[(size_t)b * M + m];
    if (pr) sr += pr[(size_t)b * M + m];
    ss += ps[b];
  }
  if (rand_per_frame) sr = (double)rpf[m] * (double)n_bins_total;
  const double c = fmax(sc - sr, 0.0) / ((double)kappa * (double)dt[m] * ss);
  cval[m] = (float)fmax(c, 1e-6);
}

template <class TX>
__global__ void k_broadcast_frames(TX* x, long long n_vox, int M, const float* cval,
                                   const float* scale) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_vox * M) return;
  const int m = (int)(idx % M);
  st1(x + idx, scale ? cval[m] / scale[m] : cval[m]);
}

// ------------------------------------------------------------ launch helpers
static int check_geom(const kcs_geometry* g, int subset, int n_frames) {
  KCS_REQUIRE(g != nullptr, "geometry is NULL");
  KCS_REQUIRE(subset >= -1 && subset < g->S, "subset %d outside [-1, %d)", subset, g->S);
  KCS_REQUIRE(n_frames >= 4 && n_frames <= 32 && n_frames % 4 == 0,
              "n_frames=%d must be a multiple of 4 in [4, 32]", n_frames);
  return KCS_OK;
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }
// a float array on 16 bytes, a 16-bit one on 8
static bool aligned_for(const void* ptr, int t) {
  return ((uintptr_t)ptr & (t == KCS_F32 ? 15u : 7u)) == 0;
}
// Quads per bin row of the ratio kept in the OSL workspace: float rows get an
// odd number of 16-byte quads so that the back-projection's 128-bit reads of
// up to 8 consecutive bins fall in distinct shared-memory bank groups (a
// 96-byte pitch repeats them every 4 bins); 16-bit rows stay dense.
static int rho_pitch(int MQ, int x_type) { return x_type == KCS_F32 ? (MQ | 1) : MQ; }

static ProjArgs base_args(const kcs_geometry* g, int subset) {
  ProjArgs p{};
  p.pair_all = g->pair_all;
  p.ang = g->d_ang;
  p.sub = subset_dev(g, subset);
  p.n_sub = subset_count(g, subset);
  p.nx = g->nx; p.ny = g->ny; p.nz = g->nz; p.B = g->B; p.A = g->A;
  const int a0 = subset < 0 ? 0 : g->off[subset], a1 = subset < 0 ? g->A : g->off[subset + 1];
  for (int i = a0; i < a1; ++i) {
    const AngleTab& T = g->h_tab[subset < 0 ? i : g->h_angles[i]];
    p.max_beta = std::max(p.max_beta, std::fabs(T.beta));
    p.max_gamma = std::max(p.max_gamma, std::fabs(T.gamma));
  }
  return p;
}

// The staged forward is built but off: measured at full size (PR2, float32)
// it takes 3.28 ms per subset against 1.49 ms for k_forward, bit-identical.
// Each block re-stages a window overlapping its neighbours' (more bytes from
// L2 than the L1 misses of k_forward) and waits for its copies at every chunk
// with fewer warps per SM.  Build with -DKCS_FWD_STAGED=1 to select it.
#ifndef KCS_FWD_STAGED
#define KCS_FWD_STAGED 0
#endif
constexpr size_t SF_SMEM_MAX = 200 * 1024;

template <int MQ, bool RATIO, class TC, class TY>
static bool launch_forward_staged(const ProjArgs& p, cudaStream_t s) {
  constexpr int R = SF_WARPS * (32 / MQ), M = 4 * MQ;
  StagedDims d;
  d.span = (int)std::ceil((double)p.max_beta * (R - 1) + (double)p.max_gamma * (SF_T - 1)) + 5;
  d.xpitch = SF_T * M + (((M - SF_T * M) % 32) + 32) % 32;   // = M (mod 32), a multiple of 4
  d.buf = std::max(SF_T * d.span * M, d.span * d.xpitch);
  const size_t smem = 2 * (size_t)d.buf * sizeof(float);
  if (smem > SF_SMEM_MAX) return false;
  auto kern = k_forward_staged<MQ, RATIO, TC, TY>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return false;
  const long long blocks = (long long)p.nz * p.n_sub * ((p.B + R - 1) / R);
  kern<<<(unsigned)blocks, SF_WARPS * 32, smem, s>>>(p, d);
  return true;
}

template <bool RATIO, class TX, class TC, class TY>
static void launch_forward_t(int MQ, const ProjArgs& p0, cudaStream_t s) {
  ProjArgs p = p0;
  if (!p.yq) p.yq = MQ;
  if (KCS_FWD_STAGED && std::is_same<TX, float>::value) {
    bool done = false;
    switch (MQ) {
      case 1: done = launch_forward_staged<1, RATIO, TC, TY>(p, s); break;
      case 2: done = launch_forward_staged<2, RATIO, TC, TY>(p, s); break;
      case 3: done = launch_forward_staged<3, RATIO, TC, TY>(p, s); break;
      case 4: done = launch_forward_staged<4, RATIO, TC, TY>(p, s); break;
      case 5: done = launch_forward_staged<5, RATIO, TC, TY>(p, s); break;
      case 6: done = launch_forward_staged<6, RATIO, TC, TY>(p, s); break;
      case 7: done = launch_forward_staged<7, RATIO, TC, TY>(p, s); break;
      case 8: done = launch_forward_staged<8, RATIO, TC, TY>(p, s); break;
    }
    if (done) return;
  }
  const int rpw = 32 / MQ;
  const long long rays = (long long)p.nz * p.n_sub * p.B;
  const long long warps = (rays + rpw - 1) / rpw;
  constexpr int wpb = FWD_THREADS / 32;
  const unsigned blocks = (unsigned)((warps + wpb - 1) / wpb);
  switch (MQ) {
    case 1: k_forward<1, RATIO, TX, TC, TY><<<blocks, FWD_THREADS, 0, s>>>(p); break;
    case 2: k_forward<2, RATIO, TX, TC, TY><<<blocks, FWD_THREADS, 0, s>>>(p); break;
    case 3: k_forward<3, RATIO, TX, TC, TY><<<blocks, FWD_THREADS, 0, s>>>(p); break;
    case 4: k_forward<4, RATIO, TX, TC, TY><<<blocks, FWD_THREADS, 0, s>>>(p); break;
    case 5: k_forward<5, RATIO, TX, TC, TY><<<blocks, FWD_THREADS, 0, s>>>(p); break;
    case 6: k_forward<6, RATIO, TX, TC, TY><<<blocks, FWD_THREADS, 0, s>>>(p); break;
    case 7: k_forward<7, RATIO, TX, TC, TY><<<blocks, FWD_THREADS, 0, s>>>(p); break;
    case 8: k_forward<8, RATIO, TX, TC, TY><<<blocks, FWD_THREADS, 0, s>>>(p); break;
  }
}

// Plain forward projection (float image -> float sinogram).
static void launch_forward(int MQ, const ProjArgs& p, cudaStream_t s) {
  launch_forward_t<false, float, float, float>(MQ, p, s);
}

// Plain forward projection of an image stored as tx (float sinogram out).
static void launch_forward_x(int MQ, int tx, const ProjArgs& p, cudaStream_t s) {
  if (tx == KCS_BF16) launch_forward_t<false, __nv_bfloat16, float, float>(MQ, p, s);
  else if (tx == KCS_F16) launch_forward_t<false, __half, float, float>(MQ, p, s);
  else launch_forward_t<false, float, float, float>(MQ, p, s);
}

// Forward + ratio with a stored image of type tx (the ratio is stored the same
// way) and counts of type tc.
template <class TX>
static void launch_ratio_tx(int MQ, int tc, const ProjArgs& p, cudaStream_t s) {
  if (tc == KCS_U16) launch_forward_t<true, TX, uint16_t, TX>(MQ, p, s);
  else launch_forward_t<true, TX, float, TX>(MQ, p, s);
}
static void launch_ratio(int MQ, int tx, int tc, const ProjArgs& p, cudaStream_t s) {
  if (tx == KCS_BF16) launch_ratio_tx<__nv_bfloat16>(MQ, tc, p, s);
  else if (tx == KCS_F16) launch_ratio_tx<__half>(MQ, tc, p, s);
  else launch_ratio_tx<float>(MQ, tc, p, s);
}

// Rows of one angle a 16 x 16 tile can touch: over the tile's corners the
// continuous bin coordinate moves by 15 (|cos| + |sin|) <= 15 sqrt(2) voxels
// and the +-1 interpolation band adds 2 (in bins: times vox / bin); the floor
// and ceiling, the margins of bin_range and the union add at most 7 rows.
static int back_rows_max(const kcs_geometry* g) {
  const double span = (BK_TILE - 1) * 1.41421357 + 2.0;
  return (int)std::ceil(span * g->vox / g->bin) + 8;
}

constexpr size_t BK_SMEM_MAX = 200 * 1024;   // dynamic shared memory budget per block

#ifndef KCS_BACK_BULK
#define KCS_BACK_BULK 1
#endif

template <int MQ, int MODE, class TX, class TY>
static int launch_back_mq(const ProjArgs& p0, int rows_max, cudaStream_t s) {
  ProjArgs p = p0;
  if (!p.yq) p.yq = MQ;
  p.aligned32 = (((uintptr_t)p.x | (uintptr_t)p.xout | (uintptr_t)p.F) & 31u) == 0;
  if (KCS_BACK_BULK && (p.yq * 4 * sizeof(TY)) % 16 == 0) {
    const size_t row_bytes = (size_t)p.yq * 4 * sizeof(TY) * rows_max;
    const int achunk = (int)std::min<size_t>(BK_ACHUNK, BK_SMEM_MAX / row_bytes);
    KCS_REQUIRE(achunk >= 1, "bins are too fine relative to voxels for the tiled back-projection");
    const size_t smem = row_bytes * achunk;
    const long long tiles = (long long)((p.nx + BK_TILE - 1) / BK_TILE) *
                            ((p.ny + BK_TILE - 1) / BK_TILE) * p.nz;
    // the OSL update with every angle under the pair rule takes the
    // two-candidate instance; everything else the general candidate loop
    auto kern = k_back_bulk<MQ, MODE, TX, TY, false>;
    if constexpr (MODE == 1)
      if (p.pair_all) kern = k_back_bulk<MQ, MODE, TX, TY, true>;
    KCS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)tiles, BK_TILE * BK_TILE, smem, s>>>(p, rows_max, achunk);
    return KCS_OK;
  }
  const size_t row_bytes = sizeof(float4) * rows_max * bk_pitch(MQ);
  const int achunk = (int)std::min<size_t>(BK_ACHUNK, BK_SMEM_MAX / row_bytes);
  KCS_REQUIRE(achunk >= 1, "bins are too fine relative to voxels for the tiled back-projection");
  const size_t smem = row_bytes * achunk;
  KCS_CUDA(cudaFuncSetAttribute(k_back_tiled<MQ, MODE, TX, TY>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const long long tiles = (long long)((p.nx + BK_TILE - 1) / BK_TILE) *
                          ((p.ny + BK_TILE - 1) / BK_TILE) * p.nz;
  k_back_tiled<MQ, MODE, TX, TY><<<(unsigned)tiles, BK_TILE * BK_TILE, smem, s>>>(p, rows_max,
                                                                                achunk);
  return KCS_OK;
}

template <int MODE, class TX, class TY>
static int launch_back_t(int MQ, const ProjArgs& p, int rows_max, cudaStream_t s) {
  switch (MQ) {
    case 1: return launch_back_mq<1, MODE, TX, TY>(p, rows_max, s);
    case 2: return launch_back_mq<2, MODE, TX, TY>(p, rows_max, s);
    case 3: return launch_back_mq<3, MODE, TX, TY>(p, rows_max, s);
    case 4: return launch_back_mq<4, MODE, TX, TY>(p, rows_max, s);
    case 5: return launch_back_mq<5, MODE, TX, TY>(p, rows_max, s);
    case 6: return launch_back_mq<6, MODE, TX, TY>(p, rows_max, s);
    case 7: return launch_back_mq<7, MODE, TX, TY>(p, rows_max, s);
    case 8: return launch_back_mq<8, MODE, TX, TY>(p, rows_max, s);
  }
  return KCS_ERR_INVALID_ARG;
}

// MODE 0: float sinogram -> float image.  MODE 1: OSL update of an image stored
// as tx from a ratio stored the same way.
// MODE 0: tx is the storage type of the sinogram y (the image out is float).
template <int MODE>
static int launch_back(int MQ, int tx, const ProjArgs& p, int rows_max, cudaStream_t s) {
  if (MODE == 0) {
    if (tx == KCS_BF16) return launch_back_t<0, float, __nv_bfloat16>(MQ, p, rows_max, s);
    if (tx == KCS_F16) return launch_back_t<0, float, __half>(MQ, p, rows_max, s);
    return launch_back_t<0, float, float>(MQ, p, rows_max, s);
  }
  if (tx == KCS_BF16) return launch_back_t<MODE, __nv_bfloat16, __nv_bfloat16>(MQ, p, rows_max, s);
  if (tx == KCS_F16) return launch_back_t<MODE, __half, __half>(MQ, p, rows_max, s);
  return launch_back_t<MODE, float, float>(MQ, p, rows_max, s);
}

}  // namespace kcs

using namespace kcs;

extern "C" {

const char* kcs_last_error(void) { return kcs::g_err.c_str(); }
int kcs_version(void) { return 3; }

int kcs_create_geometry(kcs_geometry_t** out, int nx, int ny, int nz, float vox_mm, int n_bins,
                        int n_angles, float bin_mm, int n_subsets) {
  const int st = kcs_create_geometry_ex(out, nx, ny, nz, vox_mm, n_bins, n_angles, bin_mm,
                                        n_subsets, nullptr);
  if (st == KCS_OK) {
    const cudaError_t e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) {
      kcs_destroy_geometry(*out);
      *out = nullptr;
      set_error("geometry tables: %s", cudaGetErrorString(e));
      return KCS_ERR_CUDA;
    }
  }
  return st;
}

int kcs_create_geometry_ex(kcs_geometry_t** out, int nx, int ny, int nz, float vox_mm,
                           int n_bins, int n_angles, float bin_mm, int n_subsets, void* stream) {
  clear_error();
  KCS_REQUIRE(out != nullptr, "out is NULL");
  KCS_REQUIRE(nx > 0 && ny > 0 && nz > 0 && n_bins > 0 && n_angles > 0,
              "sizes must be positive (nx=%d ny=%d nz=%d B=%d A=%d)", nx, ny, nz, n_bins, n_angles);
  KCS_REQUIRE(n_subsets > 0 && n_subsets <= n_angles, "n_subsets=%d outside [1, %d]", n_subsets,
              n_angles);
  KCS_REQUIRE(vox_mm > 0.f && bin_mm > 0.f, "voxel and bin sizes must be positive");
  KCS_REQUIRE((long long)nx * ny * 32 < (1LL << 31) && (long long)n_bins * n_angles * 32 < (1LL << 31),
              "plane too large for 32-bit in-plane offsets");
  std::vector<AngleTab> tab(n_angles);
  const double pi = 3.14159265358979323846;
  for (int a = 0; a < n_angles; ++a) {
    const double th = a * pi / n_angles;
    const double c = cos(th), s = sin(th);
    AngleTab T;
    T.xmajor = (n_angles <= 4 * a && 4 * a <= 3 * n_angles) ? 1 : 0;
    if (T.xmajor) {
      T.beta = (float)(bin_mm / (s * vox_mm));
      T.gamma = (float)(-c / s);
      T.w = (float)(vox_mm / fabs(s));
      T.inv_beta = (float)(s * vox_mm / bin_mm);
    } else {
      T.beta = (float)(bin_mm / (c * vox_mm));
      T.gamma = (float)(-s / c);
      T.w = (float)(vox_mm / fabs(c));
      T.inv_beta = (float)(c * vox_mm / bin_mm);
    }
    const int n_major = T.xmajor ? nx : ny, n_minor = T.xmajor ? ny : nx;
    T.tc = 0.5f * (float)(n_major - 1);      // the kernels' own float expressions
    T.centre = 0.5f * (float)(n_minor - 1);
    T.rband = fabsf(T.inv_beta) + 1e-3f;
    // Pair rule: a voxel at minor index m receives weight from the rays whose
    // sample lies in (m - 1, m + 1).  Consecutive bins' samples are |beta|
    // apart before rounding and each is rounded once (one fused multiply-add,
    // error <= half an ulp of |fr| < n_minor + 1), so when |beta| - 1 exceeds
    // one such ulp at most two samples fit in that open interval, on
    // consecutive bins.  |beta| = 1 with an inner position that is exactly the
    // minor centre for every major step (|gamma| (n_major - 1) / 2 below a
    // quarter ulp of the centre) makes every sample position an exact
    // half-integer sum, with the same conclusion.
    {
      const float lim = (float)(n_minor + 1);
      const float ulp = nextafterf(lim, 2.f * lim) - lim;
      const float ab = fabsf(T.beta);
      const float cen_ulp = nextafterf(T.centre + 1.f, 1e30f) - (T.centre + 1.f);
      const bool exact1 = ab == 1.f && fabsf(T.gamma) * (0.5f * (float)n_major) < 0.25f * cen_ulp;
      T.pair = (ab - 1.f > ulp || exact1) ? 1 : 0;
    }
    T.pad_[0] = T.pad_[1] = T.pad_[2] = 0;
    tab[a] = T;
  }
  int pair_all = 1;
  for (const AngleTab& T : tab) pair_all &= T.pair;
  kcs_geometry* g = new kcs_geometry();
  g->nx = nx; g->ny = ny; g->nz = nz; g->B = n_bins; g->A = n_angles; g->S = n_subsets;
  g->vox = vox_mm; g->bin = bin_mm;
  g->pair_all = pair_all;
  cudaGetDevice(&g->device);
  g->off.assign(n_subsets + 1, 0);
  for (int k = 0; k < n_subsets; ++k) {
    for (int a = k; a < n_angles; a += n_subsets) g->h_angles.push_back(a);
    g->off[k + 1] = (int)g->h_angles.size();
  }
  g->max_sub = 0;
  for (int k = 0; k < n_subsets; ++k) g->max_sub = std::max(g->max_sub, g->off[k + 1] - g->off[k]);
  for (int a = 0; a < n_angles; ++a) g->h_angles.push_back(a);
  g->d_ang = nullptr;
  g->d_angles = nullptr;
  // the host tables live in the geometry, so the copies may stay asynchronous
  g->h_tab = tab;
  cudaStream_t s = as_stream(stream);
  cudaError_t e = cudaMalloc(&g->d_ang, sizeof(AngleTab) * n_angles);
  if (e == cudaSuccess) e = cudaMalloc(&g->d_angles, sizeof(int) * g->h_angles.size());
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->d_ang, g->h_tab.data(), sizeof(AngleTab) * n_angles,
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->d_angles, g->h_angles.data(), sizeof(int) * g->h_angles.size(),
                        cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    set_error("geometry tables: %s", cudaGetErrorString(e));
    cudaFree(g->d_ang);
    cudaFree(g->d_angles);
    delete g;
    return e == cudaErrorMemoryAllocation ? KCS_ERR_OOM : KCS_ERR_CUDA;
  }
  *out = g;
  return KCS_OK;
}

int kcs_destroy_geometry(kcs_geometry_t* g) {
  clear_error();
  if (!g) return KCS_OK;
  cudaFree(g->d_ang);
  cudaFree(g->d_angles);
  delete g;
  return KCS_OK;
}

int kcs_geometry_subset_angles(const kcs_geometry_t* g, int subset, int* angles_out, int* n_out) {
  clear_error();
  KCS_REQUIRE(g != nullptr && n_out != nullptr, "NULL argument");
  KCS_REQUIRE(subset >= -1 && subset < g->S, "subset %d outside [-1, %d)", subset, g->S);
  const int n = subset_count(g, subset);
  *n_out = n;
  if (angles_out) {
    const int o = subset < 0 ? g->A : g->off[subset];
    for (int i = 0; i < n; ++i) angles_out[i] = g->h_angles[o + i];
  }
  return KCS_OK;
}

int kcs_forward_project(const kcs_geometry_t* g, int subset, int n_frames, const float* x,
                        float* y, void* stream) {
  clear_error();
  int st = check_geom(g, subset, n_frames);
  if (st) return st;
  KCS_REQUIRE(x && y, "x and y must be device pointers");
  KCS_REQUIRE(aligned16(x) && aligned16(y), "arrays must be 16-byte aligned");
  ProjArgs p = base_args(g, subset);
  p.x = x;
  p.yout = y;
  launch_forward(n_frames / 4, p, as_stream(stream));
  KCS_LAUNCHED();
  return KCS_OK;
}

int kcs_forward_project_ex(const kcs_geometry_t* g, int subset, int n_frames, const void* x,
                           int x_type, const float* x_scale, float* y, void* stream) {
  clear_error();
  int st = check_geom(g, subset, n_frames);
  if (st) return st;
  KCS_REQUIRE(x_type == KCS_F32 || x_type == KCS_BF16 || x_type == KCS_F16,
              "x_type %d must be KCS_F32, KCS_BF16 or KCS_F16", x_type);
  KCS_REQUIRE(x && y, "x and y must be device pointers");
  KCS_REQUIRE(aligned_for(x, x_type) && aligned16(y) && aligned16(x_scale),
              "x must be 16-byte (float) or 8-byte (16-bit) aligned; y and x_scale 16-byte");
  ProjArgs p = base_args(g, subset);
  p.x = x;
  p.xscale = reinterpret_cast<const float4*>(x_scale);
  p.yout = y;
  launch_forward_x(n_frames / 4, x_type, p, as_stream(stream));
  KCS_LAUNCHED();
  return KCS_OK;
}

int kcs_back_project_ex(const kcs_geometry_t* g, int subset, int n_frames, const void* y,
                        int y_type, const float* y_scale, float* x, void* stream) {
  clear_error();
  int st = check_geom(g, subset, n_frames);
  if (st) return st;
  KCS_REQUIRE(y_type == KCS_F32 || y_type == KCS_BF16 || y_type == KCS_F16,
              "y_type %d must be KCS_F32, KCS_BF16 or KCS_F16", y_type);
  KCS_REQUIRE(x && y, "x and y must be device pointers");
  KCS_REQUIRE(aligned_for(y, y_type) && aligned16(x) && aligned16(y_scale),
              "y must be 16-byte (float) or 8-byte (16-bit) aligned; x and y_scale 16-byte");
  ProjArgs p = base_args(g, subset);
  p.y = y;
  p.yscale = reinterpret_cast<const float4*>(y_scale);
  p.xout = x;
  st = launch_back<0>(n_frames / 4, y_type, p, back_rows_max(g), as_stream(stream));
  if (st) return st;
  KCS_LAUNCHED();
  return KCS_OK;
}

int kcs_back_project(const kcs_geometry_t* g, int subset, int n_frames, const float* y, float* x,
                     void* stream) {
  clear_error();
  int st = check_geom(g, subset, n_frames);
  if (st) return st;
  KCS_REQUIRE(x && y, "x and y must be device pointers");
  KCS_REQUIRE(aligned16(x) && aligned16(y), "arrays must be 16-byte aligned");
  ProjArgs p = base_args(g, subset);
  p.y = y;
  p.xout = x;
  st = launch_back<0>(n_frames / 4, KCS_F32, p, back_rows_max(g), as_stream(stream));
  if (st) return st;
  KCS_LAUNCHED();
  return KCS_OK;
}

int kcs_sensitivity(const kcs_geometry_t* g, int subset, const float* bin_factor, float* sens,
                    void* stream) {
  clear_error();
  int st = check_geom(g, subset, 4);
  if (st) return st;
  KCS_REQUIRE(sens != nullptr, "sens must be a device pointer");
  ProjArgs p = base_args(g, subset);
  p.bin_factor = bin_factor;
  const long long vox = (long long)g->nz * g->ny * g->nx;
  k_sens<<<(unsigned)((vox + 255) / 256), 256, 0, as_stream(stream)>>>(p, sens);
  KCS_LAUNCHED();
  return KCS_OK;
}

size_t kcs_osl_workspace_size(const kcs_geometry_t* g, int n_frames) {
  if (!g || n_frames <= 0) return 0;
  const size_t rho = (size_t)g->nz * g->max_sub * g->B * rho_pitch(n_frames / 4, KCS_F32) * 4 *
                     sizeof(float);
  const size_t red = align256(sizeof(double) * RED_BLOCKS * (2 * (size_t)n_frames + 1)) +
                     align256(sizeof(double) * RED_BLOCKS) + align256(sizeof(float) * 32) +
                     align256((size_t)g->nz * g->ny * g->nx * sizeof(float));
  return align256(std::max(rho, red));
}

static bool storage_ok(int t) { return t == KCS_F32 || t == KCS_BF16 || t == KCS_F16; }

static int osl_ratio(const kcs_geometry_t* g, int subset, int n_frames, const float* frame_dt,
                     float kappa, const void* counts, int counts_type, const float* randoms,
                     int randoms_layout, const float* bin_factor, const void* x, int x_type,
                     const float* x_scale, void* rho, int rho_q, void* stream) {
  int st = check_geom(g, subset, n_frames);
  if (st) return st;
  KCS_REQUIRE(subset >= 0, "the ratio needs a subset index >= 0");
  KCS_REQUIRE(frame_dt && counts && x && rho, "frame_dt, counts, x and rho must be device pointers");
  KCS_REQUIRE(storage_ok(x_type), "x_type %d must be KCS_F32, KCS_BF16 or KCS_F16", x_type);
  KCS_REQUIRE(counts_type == KCS_F32 || counts_type == KCS_U16, "counts_type %d must be KCS_F32 or KCS_U16",
              counts_type);
  KCS_REQUIRE(randoms_layout >= KCS_RANDOMS_NONE && randoms_layout <= KCS_RANDOMS_FULL,
              "bad randoms_layout %d", randoms_layout);
  KCS_REQUIRE(randoms_layout == KCS_RANDOMS_NONE || randoms, "randoms pointer is NULL");
  KCS_REQUIRE(kappa > 0.f, "kappa must be positive");
  KCS_REQUIRE(aligned_for(x, x_type) && aligned_for(rho, x_type) &&
              aligned_for(counts, counts_type == KCS_U16 ? KCS_BF16 : KCS_F32) && aligned16(frame_dt) &&
              aligned16(randoms) && aligned16(x_scale), "arrays misaligned (16 B for float, 8 B for 16-bit)");
  ProjArgs p = base_args(g, subset);
  p.x = x;
  p.xscale = reinterpret_cast<const float4*>(x_scale);
  p.yout = rho;
  p.yq = rho_q;
  p.counts = counts;
  p.randoms = reinterpret_cast<const float4*>(randoms);
  p.randoms_layout = randoms_layout;
  p.bin_factor = bin_factor;
  p.dt = reinterpret_cast<const float4*>(frame_dt);
  p.kappa = kappa;
  launch_ratio(n_frames / 4, x_type, counts_type, p, as_stream(stream));
  KCS_LAUNCHED();
  return KCS_OK;
}

int kcs_loglik(const kcs_geometry_t* g, int n_frames, const float* frame_dt, float kappa,
               const void* counts, int counts_type, const float* randoms, int randoms_layout,
               const float* bin_factor, const void* x, int x_type, const float* x_scale,
               double* out, void* workspace, size_t ws_bytes, void* stream) {
  clear_error();
  int st = check_geom(g, -1, n_frames);
  if (st) return st;
  KCS_REQUIRE(frame_dt && counts && x && out, "frame_dt, counts, x and out must be device pointers");
  KCS_REQUIRE(storage_ok(x_type), "x_type %d must be KCS_F32, KCS_BF16 or KCS_F16", x_type);
  KCS_REQUIRE(counts_type == KCS_F32 || counts_type == KCS_U16, "counts_type %d must be KCS_F32 or KCS_U16",
              counts_type);
  KCS_REQUIRE(randoms_layout >= KCS_RANDOMS_NONE && randoms_layout <= KCS_RANDOMS_FULL,
              "bad randoms_layout %d", randoms_layout);
  KCS_REQUIRE(randoms_layout == KCS_RANDOMS_NONE || randoms, "randoms pointer is NULL");
  KCS_REQUIRE(kappa > 0.f, "kappa must be positive");
  KCS_REQUIRE(workspace && ws_bytes >= sizeof(double) * LL_PARTS, "workspace too small");
  KCS_REQUIRE(aligned_for(x, x_type) &&
              aligned_for(counts, counts_type == KCS_U16 ? KCS_BF16 : KCS_F32) && aligned16(frame_dt) &&
              aligned16(randoms) && aligned16(x_scale), "arrays misaligned (16 B for float, 8 B for 16-bit)");
  cudaStream_t s = as_stream(stream);
  double* parts = static_cast<double*>(workspace);
  KCS_CUDA(cudaMemsetAsync(parts, 0, sizeof(double) * LL_PARTS, s));
  ProjArgs p = base_args(g, -1);
  p.x = x;
  p.xscale = reinterpret_cast<const float4*>(x_scale);
  p.counts = counts;
  p.randoms = reinterpret_cast<const float4*>(randoms);
  p.randoms_layout = randoms_layout;
  p.bin_factor = bin_factor;
  p.dt = reinterpret_cast<const float4*>(frame_dt);
  p.kappa = kappa;
  p.ll_partial = parts;
  launch_ratio(n_frames / 4, x_type, counts_type, p, s);
  KCS_LAUNCHED();
  k_sum_parts<<<1, 256, 0, s>>>(parts, LL_PARTS, out);
  KCS_LAUNCHED();
  return KCS_OK;
}

int kcs_osl_ratio(const kcs_geometry_t* g, int subset, int n_frames, const float* frame_dt,
                  float kappa, const float* counts, const float* randoms, int randoms_layout,
                  const float* bin_factor, const float* x, float* rho, void* stream) {
  return kcs_osl_ratio_ex(g, subset, n_frames, frame_dt, kappa, counts, KCS_F32, randoms,
                          randoms_layout, bin_factor, x, KCS_F32, nullptr, rho, n_frames, stream);
}

static int osl_backproject(const kcs_geometry_t* g, int subset, int n_frames,
                           const float* frame_dt, float kappa, const float* bin_factor,
                           const void* rho, int rho_q, const float* F_model, float beta_kp,
                           float sigma2, void* x, int x_type, const float* x_scale, void* stream) {
  int st = check_geom(g, subset, n_frames);
  if (st) return st;
  KCS_REQUIRE(subset >= 0, "the OSL update needs a subset index >= 0");
  KCS_REQUIRE(frame_dt && rho && x, "frame_dt, rho and x must be device pointers");
  KCS_REQUIRE(storage_ok(x_type), "x_type %d must be KCS_F32, KCS_BF16 or KCS_F16", x_type);
  KCS_REQUIRE(kappa > 0.f, "kappa must be positive");
  KCS_REQUIRE(!F_model || beta_kp == 0.f || sigma2 > 0.f, "sigma2 must be positive");
  KCS_REQUIRE(aligned_for(x, x_type) && aligned_for(rho, x_type) && aligned16(frame_dt) &&
              aligned16(F_model) && aligned16(x_scale), "arrays misaligned");
  ProjArgs q = base_args(g, subset);
  q.x = x;
  q.xscale = reinterpret_cast<const float4*>(x_scale);
  q.y = rho;
  q.yq = rho_q;
  q.xout = x;
  q.bin_factor = bin_factor;
  q.dt = reinterpret_cast<const float4*>(frame_dt);
  q.kappa = kappa;
  q.F = (F_model && beta_kp != 0.f) ? reinterpret_cast<const float4*>(F_model) : nullptr;
  q.prior_scale = q.F ? beta_kp / ((float)g->S * sigma2) : 0.f;
  st = launch_back<1>(n_frames / 4, x_type, q, back_rows_max(g), as_stream(stream));
  if (st) return st;
  KCS_LAUNCHED();
  return KCS_OK;
}

int kcs_osl_rho_frames(int n_frames, int x_type) {
  if (n_frames <= 0 || n_frames % 4) return n_frames;
  return 4 * rho_pitch(n_frames / 4, x_type);
}

static int check_rho_frames(int n_frames, int rho_frames) {
  KCS_REQUIRE(rho_frames >= n_frames && rho_frames % 4 == 0 && rho_frames <= 4 * 64,
              "rho_frames %d must be a multiple of 4 in [n_frames=%d, 256]", rho_frames, n_frames);
  return KCS_OK;
}

int kcs_osl_ratio_ex(const kcs_geometry_t* g, int subset, int n_frames, const float* frame_dt,
                     float kappa, const void* counts, int counts_type, const float* randoms,
                     int randoms_layout, const float* bin_factor, const void* x, int x_type,
                     const float* x_scale, void* rho, int rho_frames, void* stream) {
  clear_error();
  const int st = check_rho_frames(n_frames, rho_frames);
  if (st) return st;
  return osl_ratio(g, subset, n_frames, frame_dt, kappa, counts, counts_type, randoms,
                   randoms_layout, bin_factor, x, x_type, x_scale, rho, rho_frames / 4, stream);
}

int kcs_osl_backproject_ex(const kcs_geometry_t* g, int subset, int n_frames,
                           const float* frame_dt, float kappa, const float* bin_factor,
                           const void* rho, int rho_frames, const float* F_model, float beta_kp,
                           float sigma2, void* x, int x_type, const float* x_scale,
                           void* stream) {
  clear_error();
  const int st = check_rho_frames(n_frames, rho_frames);
  if (st) return st;
  return osl_backproject(g, subset, n_frames, frame_dt, kappa, bin_factor, rho, rho_frames / 4,
                         F_model, beta_kp, sigma2, x, x_type, x_scale, stream);
}

int kcs_osl_backproject(const kcs_geometry_t* g, int subset, int n_frames, const float* frame_dt,
                        float kappa, const float* bin_factor, const float* rho,
                        const float* F_model, float beta_kp, float sigma2, float* x,
                        void* stream) {
  return kcs_osl_backproject_ex(g, subset, n_frames, frame_dt, kappa, bin_factor, rho, n_frames,
                                F_model, beta_kp, sigma2, x, KCS_F32, nullptr, stream);
}

int kcs_osl_update_ex(const kcs_geometry_t* g, int subset, int n_frames, const float* frame_dt,
                      float kappa, const void* counts, int counts_type, const float* randoms,
                      int randoms_layout, const float* bin_factor, const float* F_model,
                      float beta_kp, float sigma2, void* x, int x_type, const float* x_scale,
                      void* workspace, size_t ws_bytes, void* stream) {
  clear_error();
  int st = check_geom(g, subset, n_frames);
  if (st) return st;
  KCS_REQUIRE(workspace && ws_bytes >= kcs_osl_workspace_size(g, n_frames),
              "workspace too small (%zu < %zu)", ws_bytes, kcs_osl_workspace_size(g, n_frames));
  const int rq = rho_pitch(n_frames / 4, x_type);
  st = osl_ratio(g, subset, n_frames, frame_dt, kappa, counts, counts_type, randoms,
                 randoms_layout, bin_factor, x, x_type, x_scale, workspace, rq, stream);
  if (st) return st;
  return osl_backproject(g, subset, n_frames, frame_dt, kappa, bin_factor, workspace, rq,
                         F_model, beta_kp, sigma2, x, x_type, x_scale, stream);
}

int kcs_osl_update(const kcs_geometry_t* g, int subset, int n_frames, const float* frame_dt,
                   float kappa, const float* counts, const float* randoms, int randoms_layout,
                   const float* bin_factor, const float* F_model, float beta_kp, float sigma2,
                   float* x, void* workspace, size_t ws_bytes, void* stream) {
  return kcs_osl_update_ex(g, subset, n_frames, frame_dt, kappa, counts, KCS_F32, randoms,
                           randoms_layout, bin_factor, F_model, beta_kp, sigma2, x, KCS_F32,
                           nullptr, workspace, ws_bytes, stream);
}

}  // extern "C"

// Per-frame level c_m of the uniform start image into cval [M] (device).
static int init_level(const kcs_geometry_t* g, int n_frames, const float* frame_dt, float kappa,
                      const void* counts, int counts_type, const float* randoms,
                      int randoms_layout, const float* bin_factor, float* cval, void* workspace,
                      size_t ws_bytes, cudaStream_t s) {
  int st = check_geom(g, -1, n_frames);
  if (st) return st;
  KCS_REQUIRE(frame_dt && counts && cval, "frame_dt, counts and the output must be device pointers");
  KCS_REQUIRE(counts_type == KCS_F32 || counts_type == KCS_U16, "counts_type must be KCS_F32 or KCS_U16");
  KCS_REQUIRE(randoms_layout >= KCS_RANDOMS_NONE && randoms_layout <= KCS_RANDOMS_FULL,
              "bad randoms_layout %d", randoms_layout);
  KCS_REQUIRE(randoms_layout == KCS_RANDOMS_NONE || randoms, "randoms pointer is NULL");
  KCS_REQUIRE(kappa > 0.f, "kappa must be positive");
  KCS_REQUIRE(workspace && ws_bytes >= kcs_osl_workspace_size(g, n_frames), "workspace too small");
  const int M = n_frames;
  char* w = static_cast<char*>(workspace);
  double* pc = reinterpret_cast<double*>(w);
  double* pr = pc + (size_t)RED_BLOCKS * M;
  double* ps = reinterpret_cast<double*>(w + align256(sizeof(double) * RED_BLOCKS * (2 * (size_t)M + 1)));
  float* sens = reinterpret_cast<float*>(reinterpret_cast<char*>(ps) + align256(sizeof(double) * RED_BLOCKS) +
                                         align256(sizeof(float) * 32));
  const long long n_bins_total = (long long)g->nz * g->A * g->B;
  const long long n_vox = (long long)g->nz * g->ny * g->nx;
  if (counts_type == KCS_U16)
    k_partial_sums<<<RED_BLOCKS, 256, 0, s>>>(static_cast<const uint16_t*>(counts), n_bins_total, M, pc);
  else
    k_partial_sums<<<RED_BLOCKS, 256, 0, s>>>(static_cast<const float*>(counts), n_bins_total, M, pc);
  KCS_LAUNCHED();
  if (randoms_layout == KCS_RANDOMS_FULL) {
    k_partial_sums<<<RED_BLOCKS, 256, 0, s>>>(randoms, n_bins_total, M, pr);
    KCS_LAUNCHED();
  }
  ProjArgs p = base_args(g, -1);
  p.bin_factor = bin_factor;
  k_sens<<<(unsigned)((n_vox + 255) / 256), 256, 0, s>>>(p, sens);
  KCS_LAUNCHED();
  k_partial_sums<<<RED_BLOCKS, 256, 0, s>>>(static_cast<const float*>(sens), n_vox, 1, ps);
  KCS_LAUNCHED();
  k_init_fill<<<1, 32, 0, s>>>(pc, randoms_layout == KCS_RANDOMS_FULL ? pr : nullptr, ps,
                                randoms_layout == KCS_RANDOMS_PER_FRAME, randoms, n_bins_total,
                                frame_dt, kappa, M, cval);
  KCS_LAUNCHED();
  return KCS_OK;
}

extern "C" {

int kcs_init_level(const kcs_geometry_t* g, int n_frames, const float* frame_dt, float kappa,
                   const void* counts, int counts_type, const float* randoms, int randoms_layout,
                   const float* bin_factor, float* level, void* workspace, size_t ws_bytes,
                   void* stream) {
  clear_error();
  return init_level(g, n_frames, frame_dt, kappa, counts, counts_type, randoms, randoms_layout,
                    bin_factor, level, workspace, ws_bytes, as_stream(stream));
}

int kcs_init_image_ex(const kcs_geometry_t* g, int n_frames, const float* frame_dt, float kappa,
                      const void* counts, int counts_type, const float* randoms,
                      int randoms_layout, const float* bin_factor, void* x, int x_type,
                      const float* x_scale, void* workspace, size_t ws_bytes, void* stream) {
  clear_error();
  KCS_REQUIRE(x, "x must be a device pointer");
  KCS_REQUIRE(storage_ok(x_type), "x_type %d must be KCS_F32, KCS_BF16 or KCS_F16", x_type);
  cudaStream_t s = as_stream(stream);
  KCS_REQUIRE(g && workspace, "NULL geometry or workspace");
  char* w = static_cast<char*>(workspace);
  float* cval = reinterpret_cast<float*>(
      w + align256(sizeof(double) * RED_BLOCKS * (2 * (size_t)n_frames + 1)) +
      align256(sizeof(double) * RED_BLOCKS));
  const int st = init_level(g, n_frames, frame_dt, kappa, counts, counts_type, randoms,
                            randoms_layout, bin_factor, cval, workspace, ws_bytes, s);
  if (st) return st;
  const int M = n_frames;
  const long long n_vox = (long long)g->nz * g->ny * g->nx;
  const long long n = n_vox * M;
  const unsigned nb = (unsigned)((n + 255) / 256);
  if (x_type == KCS_BF16)
    k_broadcast_frames<<<nb, 256, 0, s>>>(static_cast<__nv_bfloat16*>(x), n_vox, M, cval, x_scale);
  else if (x_type == KCS_F16)
    k_broadcast_frames<<<nb, 256, 0, s>>>(static_cast<__half*>(x), n_vox, M, cval, x_scale);
  else
    k_broadcast_frames<<<nb, 256, 0, s>>>(static_cast<float*>(x), n_vox, M, cval, x_scale);
  KCS_LAUNCHED();
  return KCS_OK;
}

int kcs_device_status_reset(void) {
  clear_error();
  const unsigned int zero = 0;
  KCS_CUDA(cudaMemcpyToSymbol(g_wait_timeouts, &zero, sizeof zero));
  return KCS_OK;
}

int kcs_selftest_wait_timeout(int spin_limit, void* stream) {
  clear_error();
  KCS_REQUIRE(spin_limit > 0 && spin_limit <= (1 << 20), "spin_limit must be in (0, 2^20]");
  k_selftest_wait<<<1, 32, 0, as_stream(stream)>>>(spin_limit);
  KCS_LAUNCHED();
  return KCS_OK;
}

int kcs_device_status(unsigned int* wait_timeouts) {
  clear_error();
  KCS_REQUIRE(wait_timeouts, "NULL argument");
  KCS_CUDA(cudaMemcpyFromSymbol(wait_timeouts, g_wait_timeouts, sizeof(unsigned int)));
  return *wait_timeouts ? KCS_ERR_TIMEOUT : KCS_OK;
}

int kcs_init_image(const kcs_geometry_t* g, int n_frames, const float* frame_dt, float kappa,
                   const float* counts, const float* randoms, int randoms_layout,
                   const float* bin_factor, float* x, void* workspace, size_t ws_bytes,
                   void* stream) {
  return kcs_init_image_ex(g, n_frames, frame_dt, kappa, counts, KCS_F32, randoms, randoms_layout,
                           bin_factor, x, KCS_F32, nullptr, workspace, ws_bytes, stream);
}

}  // extern "C"
