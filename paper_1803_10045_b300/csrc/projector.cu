// Joseph projector, its exact transpose and the fused OS-MAP-OSL update
// (Eq. 2-3 of Scipioni et al., "Kinetic Compressive Sensing").
//
// Data layout: images [Z][ny][nx][M] and sinograms [Z][A][B][M] keep the M
// frames of one voxel / bin contiguous, so every sample of a ray moves whole
// float4 frame quads.  A warp holds 32/MQ rays (forward) or voxels (back), MQ =
// M/4 lanes each, so one load instruction fetches the contiguous frame vectors
// of several rays.  The back-projection is a gather: each voxel recomputes the
// forward's sample positions with the same fused multiply-adds, so the set of
// (voxel, bin, weight) triples is exactly the forward's, with no atomics.

#include <cstdarg>
#include <cmath>
#include <algorithm>

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

// Fractional minor index of centred bin bf given inner = fma(tf, gamma, centre)
// (shared by both kernels, explicit fused multiply-adds: identical bits).
__device__ __forceinline__ float minor_pos(float bf, float beta, float inner) {
  return __fmaf_rn(bf, beta, inner);
}
__device__ __forceinline__ float inner_pos(float tf, float gamma, float centre) {
  return __fmaf_rn(tf, gamma, centre);
}

struct ProjArgs {
  const float4* x;        // image (forward input / OSL in-out)
  float4* xout;           // image output (back-projection)
  const float4* y;        // subset sinogram input (back-projection)
  float4* yout;           // subset sinogram output (forward)
  const AngleTab* ang;
  const int* sub;         // angle indices of the subset
  int n_sub;
  int nx, ny, nz, B, A;
  // ratio / OSL terms
  const float4* counts;   // [Z][A][B][MQ]
  const float4* randoms;  // per frame [MQ] or full [Z][A][B][MQ]
  int randoms_layout;
  const float* bin_factor;  // [Z][A][B] or null
  const float4* dt;         // [MQ]
  float kappa;
  const float4* F;          // model TACs or null
  float prior_scale;        // beta / (S sigma2)
};

// Forward projection of every frame of rays (z, ak, b); RATIO replaces the
// projection by rho = s / (kappa dt n_d (P x) + r).
template <int MQ, bool RATIO>
__global__ void __launch_bounds__(256) k_forward(ProjArgs p) {
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
  const int s_major = T.xmajor ? MQ : p.nx * MQ;   // float4 stride of one major step
  const int s_minor = T.xmajor ? p.nx * MQ : MQ;   // float4 stride of one minor step
  const float tc = 0.5f * (float)(n_major - 1);
  const float centre = 0.5f * (float)(n_minor - 1);
  const float bf = (float)b - 0.5f * (float)(p.B - 1);
  const float4* xz = p.x + (size_t)z * p.ny * p.nx * MQ + q;

  // Conservative major-step range where the ray can touch the grid; the exact
  // test is repeated per step below.
  int t0 = 0, t1 = n_major - 1;
  const float base = __fmaf_rn(bf, T.beta, centre);
  if (fabsf(T.gamma) > 1e-6f) {
    const float ta = (-1.0f - base) / T.gamma + tc;
    const float tb = ((float)n_minor - base) / T.gamma + tc;
    const float lo = fminf(ta, tb), hi = fmaxf(ta, tb);
    t0 = max(0, (int)floorf(fmaxf(lo, -4.0f)) - 2);
    t1 = min(n_major - 1, (int)ceilf(fminf(hi, (float)n_major + 4.0f)) + 2);
  }
  float4 acc = f4(0.f);
  for (int t = t0; t <= t1; ++t) {
    const float fr = minor_pos(bf, T.beta, inner_pos((float)t - tc, T.gamma, centre));
    const float fl = floorf(fr);
    const int j0 = (int)fl;
    if (j0 < -1 || j0 >= n_minor) continue;
    const float f = fr - fl;
    const float4* px = xz + (size_t)t * s_major + (ptrdiff_t)j0 * s_minor;
    if (j0 >= 0) fma4(acc, 1.0f - f, __ldg(px));
    if (j0 + 1 < n_minor) fma4(acc, f, __ldg(px + s_minor));
  }
  acc.x *= T.w; acc.y *= T.w; acc.z *= T.w; acc.w *= T.w;
  const size_t oi = ((size_t)(z * p.n_sub + ak) * p.B + b) * MQ + q;
  if (!RATIO) {
    p.yout[oi] = acc;
    return;
  }
  const size_t bin = (size_t)(z * p.A + a) * p.B + b;
  const float nd = p.bin_factor ? __ldg(p.bin_factor + bin) : 1.0f;
  const float4 dt = __ldg(p.dt + q);
  const float4 s = __ldg(p.counts + bin * MQ + q);
  float4 r = f4(0.f);
  if (p.randoms_layout == KCS_RANDOMS_PER_FRAME) r = __ldg(p.randoms + q);
  else if (p.randoms_layout == KCS_RANDOMS_FULL) r = __ldg(p.randoms + bin * MQ + q);
  const float kn = p.kappa * nd;
  float4 yb, rho;
  yb.x = fmaf(kn * dt.x, acc.x, r.x);
  yb.y = fmaf(kn * dt.y, acc.y, r.y);
  yb.z = fmaf(kn * dt.z, acc.z, r.z);
  yb.w = fmaf(kn * dt.w, acc.w, r.w);
  rho.x = yb.x > 0.f ? s.x / yb.x : 0.f;
  rho.y = yb.y > 0.f ? s.y / yb.y : 0.f;
  rho.z = yb.z > 0.f ? s.z / yb.z : 0.f;
  rho.w = yb.w > 0.f ? s.w / yb.w : 0.f;
  p.yout[oi] = rho;
}

// Bins of angle T whose sample at major step t lands within one minor step of
// m: the exact test is made per candidate by the caller.
__device__ __forceinline__ void bin_range(const AngleTab& T, int m, float inner, float bc, int B,
                                          int& b_lo, int& b_hi) {
  float lo = ((float)(m - 1) - inner) / T.beta;
  float hi = ((float)(m + 1) - inner) / T.beta;
  if (lo > hi) { const float tmp = lo; lo = hi; hi = tmp; }
  b_lo = max(0, (int)floorf(fmaxf(lo + bc, -2.0f)) - 1);
  b_hi = min(B - 1, (int)ceilf(fminf(hi + bc, (float)B + 2.0f)) + 1);
}

// Gather back-projection.  MODE 0: x = P_k^T y.  MODE 1: OSL update of x in
// place with y = rho (Eq. 2 with the prior of Eq. 3).
template <int MQ, int MODE>
__global__ void __launch_bounds__(256) k_back(ProjArgs p) {
  constexpr int VPW = 32 / MQ;
  const int lane = threadIdx.x & 31;
  const int sub = lane / MQ;
  const int q = lane - sub * MQ;
  if (sub >= VPW) return;
  const long long vox = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * VPW + sub;
  const long long n_vox = (long long)p.nz * p.ny * p.nx;
  if (vox >= n_vox) return;
  const int i = (int)(vox % p.nx);
  const long long zj = vox / p.nx;
  const int j = (int)(zj % p.ny);
  const int z = (int)(zj / p.ny);
  const float bc = 0.5f * (float)(p.B - 1);
  float4 acc = f4(0.f);
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
    bin_range(T, m, inner, bc, p.B, b_lo, b_hi);
    const float4* yrow = p.y + (size_t)(z * p.n_sub + ak) * p.B * MQ + q;
    const size_t binrow = (size_t)(z * p.A + a) * p.B;
    for (int b = b_lo; b <= b_hi; ++b) {
      const float fr = minor_pos((float)b - bc, T.beta, inner);
      const float fl = floorf(fr);
      const int j0 = (int)fl;
      const float f = fr - fl;
      float wt = (j0 == m) ? 1.0f - f : ((j0 + 1 == m) ? f : 0.0f);
      if (wt == 0.0f) continue;
      wt *= T.w;
      if (MODE == 1 && p.bin_factor) wt *= __ldg(p.bin_factor + binrow + b);
      fma4(acc, wt, __ldg(yrow + (size_t)b * MQ));
      sens += wt;
    }
  }
  const size_t vi = (size_t)vox * MQ + q;
  if (MODE == 0) {
    p.xout[vi] = acc;
    return;
  }
  float4 xv = p.x[vi];
  if (sens > 0.f) {
    const float4 dt = __ldg(p.dt + q);
    const float ks = p.kappa * sens;
    float4 den = make_float4(dt.x * ks, dt.y * ks, dt.z * ks, dt.w * ks);
    if (p.F) {
      const float4 Fv = __ldg(p.F + vi);
      const float ps = p.prior_scale;
      den.x = fmaxf(fmaf(ps, xv.x - Fv.x, den.x), 1e-3f * den.x);
      den.y = fmaxf(fmaf(ps, xv.y - Fv.y, den.y), 1e-3f * den.y);
      den.z = fmaxf(fmaf(ps, xv.z - Fv.z, den.z), 1e-3f * den.z);
      den.w = fmaxf(fmaf(ps, xv.w - Fv.w, den.w), 1e-3f * den.w);
    }
    xv.x = xv.x * (p.kappa * dt.x * acc.x) / den.x;
    xv.y = xv.y * (p.kappa * dt.y * acc.y) / den.y;
    xv.z = xv.z * (p.kappa * dt.z * acc.z) / den.z;
    xv.w = xv.w * (p.kappa * dt.w * acc.w) / den.w;
  }
  p.xout[vi] = xv;
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
    bin_range(T, m, inner, bc, p.B, b_lo, b_hi);
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

__global__ void __launch_bounds__(256) k_partial_sums(const float* data, long long n_rows, int M,
                                                      double* partial /*[RED_BLOCKS][M]*/) {
  __shared__ double sh[256];
  const int tid = threadIdx.x;
  const long long per = (n_rows + gridDim.x - 1) / gridDim.x;
  const long long r0 = (long long)blockIdx.x * per;
  const long long r1 = min(n_rows, r0 + per);
  for (int m = 0; m < M; ++m) {
    double s = 0.0;
    for (long long r = r0 + tid; r < r1; r += blockDim.x) s += (double)data[r * M + m];
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

__global__ void k_broadcast_frames(float* x, long long n_vox, int M, const float* cval) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_vox * M) return;
  x[idx] = cval[idx % M];
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

static ProjArgs base_args(const kcs_geometry* g, int subset) {
  ProjArgs p{};
  p.ang = g->d_ang;
  p.sub = subset_dev(g, subset);
  p.n_sub = subset_count(g, subset);
  p.nx = g->nx; p.ny = g->ny; p.nz = g->nz; p.B = g->B; p.A = g->A;
  return p;
}

template <bool RATIO>
static void launch_forward(int MQ, const ProjArgs& p, cudaStream_t s) {
  const int rpw = 32 / MQ;
  const long long rays = (long long)p.nz * p.n_sub * p.B;
  const long long warps = (rays + rpw - 1) / rpw;
  const unsigned blocks = (unsigned)((warps + 7) / 8);
  switch (MQ) {
    case 1: k_forward<1, RATIO><<<blocks, 256, 0, s>>>(p); break;
    case 2: k_forward<2, RATIO><<<blocks, 256, 0, s>>>(p); break;
    case 3: k_forward<3, RATIO><<<blocks, 256, 0, s>>>(p); break;
    case 4: k_forward<4, RATIO><<<blocks, 256, 0, s>>>(p); break;
    case 5: k_forward<5, RATIO><<<blocks, 256, 0, s>>>(p); break;
    case 6: k_forward<6, RATIO><<<blocks, 256, 0, s>>>(p); break;
    case 7: k_forward<7, RATIO><<<blocks, 256, 0, s>>>(p); break;
    case 8: k_forward<8, RATIO><<<blocks, 256, 0, s>>>(p); break;
  }
}

template <int MODE>
static void launch_back(int MQ, const ProjArgs& p, cudaStream_t s) {
  const int vpw = 32 / MQ;
  const long long vox = (long long)p.nz * p.ny * p.nx;
  const long long warps = (vox + vpw - 1) / vpw;
  const unsigned blocks = (unsigned)((warps + 7) / 8);
  switch (MQ) {
    case 1: k_back<1, MODE><<<blocks, 256, 0, s>>>(p); break;
    case 2: k_back<2, MODE><<<blocks, 256, 0, s>>>(p); break;
    case 3: k_back<3, MODE><<<blocks, 256, 0, s>>>(p); break;
    case 4: k_back<4, MODE><<<blocks, 256, 0, s>>>(p); break;
    case 5: k_back<5, MODE><<<blocks, 256, 0, s>>>(p); break;
    case 6: k_back<6, MODE><<<blocks, 256, 0, s>>>(p); break;
    case 7: k_back<7, MODE><<<blocks, 256, 0, s>>>(p); break;
    case 8: k_back<8, MODE><<<blocks, 256, 0, s>>>(p); break;
  }
}

}  // namespace kcs

using namespace kcs;

extern "C" {

const char* kcs_last_error(void) { return kcs::g_err.c_str(); }
int kcs_version(void) { return 1; }

int kcs_create_geometry(kcs_geometry_t** out, int nx, int ny, int nz, float vox_mm, int n_bins,
                        int n_angles, float bin_mm, int n_subsets) {
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
    } else {
      T.beta = (float)(bin_mm / (c * vox_mm));
      T.gamma = (float)(-s / c);
      T.w = (float)(vox_mm / fabs(c));
    }
    tab[a] = T;
  }
  kcs_geometry* g = new kcs_geometry();
  g->nx = nx; g->ny = ny; g->nz = nz; g->B = n_bins; g->A = n_angles; g->S = n_subsets;
  g->vox = vox_mm; g->bin = bin_mm;
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
  cudaError_t e = cudaMalloc(&g->d_ang, sizeof(AngleTab) * n_angles);
  if (e == cudaSuccess) e = cudaMalloc(&g->d_angles, sizeof(int) * g->h_angles.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(g->d_ang, tab.data(), sizeof(AngleTab) * n_angles, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(g->d_angles, g->h_angles.data(), sizeof(int) * g->h_angles.size(),
                   cudaMemcpyHostToDevice);
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
  p.x = reinterpret_cast<const float4*>(x);
  p.yout = reinterpret_cast<float4*>(y);
  launch_forward<false>(n_frames / 4, p, as_stream(stream));
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
  p.y = reinterpret_cast<const float4*>(y);
  p.xout = reinterpret_cast<float4*>(x);
  launch_back<0>(n_frames / 4, p, as_stream(stream));
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
  const size_t rho = (size_t)g->nz * g->max_sub * g->B * n_frames * sizeof(float);
  const size_t red = align256(sizeof(double) * RED_BLOCKS * (2 * (size_t)n_frames + 1)) +
                     align256(sizeof(double) * RED_BLOCKS) + align256(sizeof(float) * 32) +
                     align256((size_t)g->nz * g->ny * g->nx * sizeof(float));
  return align256(std::max(rho, red));
}

int kcs_osl_ratio(const kcs_geometry_t* g, int subset, int n_frames, const float* frame_dt,
                  float kappa, const float* counts, const float* randoms, int randoms_layout,
                  const float* bin_factor, const float* x, float* rho, void* stream) {
  clear_error();
  int st = check_geom(g, subset, n_frames);
  if (st) return st;
  KCS_REQUIRE(subset >= 0, "the ratio needs a subset index >= 0");
  KCS_REQUIRE(frame_dt && counts && x && rho, "frame_dt, counts, x and rho must be device pointers");
  KCS_REQUIRE(randoms_layout >= KCS_RANDOMS_NONE && randoms_layout <= KCS_RANDOMS_FULL,
              "bad randoms_layout %d", randoms_layout);
  KCS_REQUIRE(randoms_layout == KCS_RANDOMS_NONE || randoms, "randoms pointer is NULL");
  KCS_REQUIRE(kappa > 0.f, "kappa must be positive");
  KCS_REQUIRE(aligned16(x) && aligned16(counts) && aligned16(frame_dt) && aligned16(rho) &&
              aligned16(randoms), "arrays must be 16-byte aligned");
  ProjArgs p = base_args(g, subset);
  p.x = reinterpret_cast<const float4*>(x);
  p.yout = reinterpret_cast<float4*>(rho);
  p.counts = reinterpret_cast<const float4*>(counts);
  p.randoms = reinterpret_cast<const float4*>(randoms);
  p.randoms_layout = randoms_layout;
  p.bin_factor = bin_factor;
  p.dt = reinterpret_cast<const float4*>(frame_dt);
  p.kappa = kappa;
  launch_forward<true>(n_frames / 4, p, as_stream(stream));
  KCS_LAUNCHED();
  return KCS_OK;
}

int kcs_osl_backproject(const kcs_geometry_t* g, int subset, int n_frames, const float* frame_dt,
                        float kappa, const float* bin_factor, const float* rho,
                        const float* F_model, float beta_kp, float sigma2, float* x,
                        void* stream) {
  clear_error();
  int st = check_geom(g, subset, n_frames);
  if (st) return st;
  KCS_REQUIRE(subset >= 0, "the OSL update needs a subset index >= 0");
  KCS_REQUIRE(frame_dt && rho && x, "frame_dt, rho and x must be device pointers");
  KCS_REQUIRE(kappa > 0.f, "kappa must be positive");
  KCS_REQUIRE(!F_model || beta_kp == 0.f || sigma2 > 0.f, "sigma2 must be positive");
  KCS_REQUIRE(aligned16(x) && aligned16(rho) && aligned16(frame_dt) && aligned16(F_model),
              "arrays must be 16-byte aligned");
  ProjArgs q = base_args(g, subset);
  q.x = reinterpret_cast<const float4*>(x);
  q.y = reinterpret_cast<const float4*>(rho);
  q.xout = reinterpret_cast<float4*>(x);
  q.bin_factor = bin_factor;
  q.dt = reinterpret_cast<const float4*>(frame_dt);
  q.kappa = kappa;
  q.F = (F_model && beta_kp != 0.f) ? reinterpret_cast<const float4*>(F_model) : nullptr;
  q.prior_scale = q.F ? beta_kp / ((float)g->S * sigma2) : 0.f;
  launch_back<1>(n_frames / 4, q, as_stream(stream));
  KCS_LAUNCHED();
  return KCS_OK;
}

int kcs_osl_update(const kcs_geometry_t* g, int subset, int n_frames, const float* frame_dt,
                   float kappa, const float* counts, const float* randoms, int randoms_layout,
                   const float* bin_factor, const float* F_model, float beta_kp, float sigma2,
                   float* x, void* workspace, size_t ws_bytes, void* stream) {
  clear_error();
  int st = check_geom(g, subset, n_frames);
  if (st) return st;
  KCS_REQUIRE(workspace && ws_bytes >= kcs_osl_workspace_size(g, n_frames),
              "workspace too small (%zu < %zu)", ws_bytes, kcs_osl_workspace_size(g, n_frames));
  float* rho = static_cast<float*>(workspace);
  st = kcs_osl_ratio(g, subset, n_frames, frame_dt, kappa, counts, randoms, randoms_layout,
                     bin_factor, x, rho, stream);
  if (st) return st;
  return kcs_osl_backproject(g, subset, n_frames, frame_dt, kappa, bin_factor, rho, F_model,
                             beta_kp, sigma2, x, stream);
}

int kcs_init_image(const kcs_geometry_t* g, int n_frames, const float* frame_dt, float kappa,
                   const float* counts, const float* randoms, int randoms_layout,
                   const float* bin_factor, float* x, void* workspace, size_t ws_bytes,
                   void* stream) {
  clear_error();
  int st = check_geom(g, -1, n_frames);
  if (st) return st;
  KCS_REQUIRE(frame_dt && counts && x, "frame_dt, counts and x must be device pointers");
  KCS_REQUIRE(randoms_layout >= KCS_RANDOMS_NONE && randoms_layout <= KCS_RANDOMS_FULL,
              "bad randoms_layout %d", randoms_layout);
  KCS_REQUIRE(randoms_layout == KCS_RANDOMS_NONE || randoms, "randoms pointer is NULL");
  KCS_REQUIRE(kappa > 0.f, "kappa must be positive");
  KCS_REQUIRE(workspace && ws_bytes >= kcs_osl_workspace_size(g, n_frames), "workspace too small");
  cudaStream_t s = as_stream(stream);
  const int M = n_frames;
  char* w = static_cast<char*>(workspace);
  double* pc = reinterpret_cast<double*>(w);
  double* pr = pc + (size_t)RED_BLOCKS * M;
  double* ps = reinterpret_cast<double*>(w + align256(sizeof(double) * RED_BLOCKS * (2 * (size_t)M + 1)));
  float* cval = reinterpret_cast<float*>(reinterpret_cast<char*>(ps) + align256(sizeof(double) * RED_BLOCKS));
  float* sens = reinterpret_cast<float*>(reinterpret_cast<char*>(cval) + align256(sizeof(float) * 32));
  const long long n_bins_total = (long long)g->nz * g->A * g->B;
  const long long n_vox = (long long)g->nz * g->ny * g->nx;
  k_partial_sums<<<RED_BLOCKS, 256, 0, s>>>(counts, n_bins_total, M, pc);
  KCS_LAUNCHED();
  if (randoms_layout == KCS_RANDOMS_FULL) {
    k_partial_sums<<<RED_BLOCKS, 256, 0, s>>>(randoms, n_bins_total, M, pr);
    KCS_LAUNCHED();
  }
  ProjArgs p = base_args(g, -1);
  p.bin_factor = bin_factor;
  k_sens<<<(unsigned)((n_vox + 255) / 256), 256, 0, s>>>(p, sens);
  KCS_LAUNCHED();
  k_partial_sums<<<RED_BLOCKS, 256, 0, s>>>(sens, n_vox, 1, ps);
  KCS_LAUNCHED();
  k_init_fill<<<1, 32, 0, s>>>(pc, randoms_layout == KCS_RANDOMS_FULL ? pr : nullptr, ps,
                                randoms_layout == KCS_RANDOMS_PER_FRAME, randoms, n_bins_total,
                                frame_dt, kappa, M, cval);
  KCS_LAUNCHED();
  const long long n = n_vox * M;
  k_broadcast_frames<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, n_vox, M, cval);
  KCS_LAUNCHED();
  return KCS_OK;
}

}  // extern "C"
