// FDG two-tissue irreversible model (frame-integrated, analytic) and the MAP
// Levenberg-Marquardt fit with the Huber MRF prior (Eq. 4-6 of Scipioni et al.,
// "Kinetic Compressive Sensing"; model of Sec. III-A / IV-A).
//
// Model evaluation.  With a = k2 + k3 and the running integrals
//   I(t) = int_0^t Cp(s) e^{-a(t-s)} ds,   J(t) = int_0^t I,
// C1 = K1 I and C2 = K1 k3 J, so the frame integral of C_T is
// K1 (int I + k3 int J).  Over one interval of length D starting at ts, with
// c(u) = Cp(ts + u), every a-dependent quantity is e^{-aD} times a power series
// in a with NON-NEGATIVE coefficients, e.g.
//   int_0^D c(u) e^{-a(D-u)} du = e^{-aD} sum_n a^n int_0^D c(u) u^n / n! du,
// and likewise for int I, int J, the homogeneous terms and their a-derivatives
// (10 channels).  A series of positive terms has no cancellation, is smooth
// through a -> 0 and a -> any input exponent, and gives d/da in closed form.
// The coefficients (input moments) are tabulated once per frame schedule in
// float64 by Gauss-Legendre quadrature; each voxel then evaluates, per
// interval, one exp and Horner recurrences of K(aD) terms in float32.

#include <cmath>
#include <algorithm>
#include <mutex>

#include "kcs_internal.cuh"

namespace kcs {

// ---------------------------------------------------------------- tables
struct TabArgs {
  const double* iv_t0;   // [n_iv] interval start
  const double* iv_dt;   // [n_iv] interval length
  const double* gl_x;    // [NGL] Gauss-Legendre nodes on [-1, 1]
  const double* gl_w;    // [NGL] weights
  int n_gl, n_panel;
  double A1, A2, A3, l1, l2, l3;
  float* coef;           // [n_iv][KMAX][NCH]
  double* m0;            // [n_iv] int_0^D c(u) du
};

__device__ double feng_cp(double t, const TabArgs& a) {
  if (t < 0.0) return 0.0;
  return (a.A1 * t - a.A2 - a.A3) * exp(-a.l1 * t) + a.A2 * exp(-a.l2 * t) + a.A3 * exp(-a.l3 * t);
}

// One thread per (interval, term n).  Channel weights over u in [0, D], v = D - u:
//   m1: u^n/n!                    d1: v u^n/n!
//   m2: sum_j u^j/j! v^{n+1-j}/(n+1-j)!       d2: sum_j u^j/j! v^{n+2-j}/(n+2-j)!
//   m3: sum_j u^j/j! v^{k+2}(k+1)/(k+2)!     d3: sum_j u^j/j! v^{k+3}(k+1)/(k+3)!  (k = n-j)
// integrated against c(u); g, gp, h, hp are the input-free homogeneous terms.
__global__ void k_tabulate(TabArgs a) {
  const int iv = blockIdx.x;
  const int n = threadIdx.x;
  if (n >= KMAX) return;
  const double D = a.iv_dt[iv];
  const double t0 = a.iv_t0[iv];
  double P[KMAX + 4], Q[KMAX + 4];   // u^j/j!, v^k/k!
  double m1 = 0, d1 = 0, m2 = 0, d2 = 0, m3 = 0, d3 = 0, s0 = 0;
  const double hp = D / a.n_panel;
  for (int pnl = 0; pnl < a.n_panel; ++pnl) {
    for (int g = 0; g < a.n_gl; ++g) {
      const double u = hp * (pnl + 0.5 * (a.gl_x[g] + 1.0));
      const double wq = 0.5 * hp * a.gl_w[g];
      const double v = D - u;
      const double c = feng_cp(t0 + u, a) * wq;
      P[0] = 1.0;
      Q[0] = 1.0;
      for (int j = 1; j <= n + 3; ++j) {
        P[j] = P[j - 1] * u / j;
        Q[j] = Q[j - 1] * v / j;
      }
      double sm2 = 0, sd2 = 0, sm3 = 0, sd3 = 0;
      for (int j = 0; j <= n; ++j) {
        const int k = n - j;
        sm2 += P[j] * Q[k + 1];
        sd2 += P[j] * Q[k + 2];
        sm3 += P[j] * Q[k + 2] * (k + 1);
        sd3 += P[j] * Q[k + 3] * (k + 1);
      }
      m1 += c * P[n];
      d1 += c * v * P[n];
      m2 += c * sm2;
      d2 += c * sd2;
      m3 += c * sm3;
      d3 += c * sd3;
      s0 += c;
    }
  }
  // input-independent channels: D^{n+1}/(n+1)!, D^{n+2}/(n+2)!, D^{n+2}(n+1)/(n+2)!,
  // D^{n+3}(n+1)/(n+3)!
  double f1 = 1.0;
  for (int j = 1; j <= n + 1; ++j) f1 *= D / j;
  const double f2 = f1 * D / (n + 2);
  const double f3 = f2 * D / (n + 3);
  float* o = a.coef + ((size_t)iv * KMAX + n) * NCH;
  o[CH_M1] = (float)m1;
  o[CH_G] = (float)f1;
  o[CH_M2] = (float)m2;
  o[CH_H] = (float)(f2 * (n + 1));
  o[CH_M3] = (float)m3;
  o[CH_D1] = (float)d1;
  o[CH_GP] = (float)f2;
  o[CH_D2] = (float)d2;
  o[CH_HP] = (float)(f3 * (n + 1));
  o[CH_D3] = (float)d3;
  o[10] = 0.f;
  o[11] = 0.f;
  if (n == 0) a.m0[iv] = s0;
}

__global__ void k_frame_tables(const double* m0, const int* code, int n_iv, const double* fdt,
                               int M, float* fr_cp, float* fr_inv) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  double s = 0.0;
  for (int i = 0; i < n_iv; ++i)
    if (code[i] >= 0 && (code[i] >> 1) == m) s += m0[i];
  fr_cp[m] = (float)(s / fdt[m]);
  fr_inv[m] = (float)(1.0 / fdt[m]);
}

// ---------------------------------------------------------------- model
// Evaluates F_m (and dF_m/d(K1,k2,k3,Vb) when JAC) frame by frame and hands
// each finished frame to sink(m, F, J0, J1, J2, J3).
template <bool JAC, class Sink>
__device__ __forceinline__ void eval_model(const KinDev& kd, float K1, float k2, float k3, float Vb,
                                           Sink& sink) {
  const float a = k2 + k3;
  float I = 0.f, Ip = 0.f, Jr = 0.f, Jp = 0.f;
  float SA = 0.f, SB = 0.f, SAp = 0.f, SBp = 0.f;
  for (int iv = 0; iv < kd.n_iv; ++iv) {
    const float D = __ldg(kd.iv_dt + iv);
    const float y = a * D;
    const int K = min(KMAX, (int)ceilf(2.72f * y) + 12);
    const float4* c = kd.coef + (size_t)iv * KMAX * 3;
    // Horner from the highest term down.
    float p_m1 = 0.f, p_g = 0.f, p_m2 = 0.f, p_h = 0.f, p_m3 = 0.f;
    float p_d1 = 0.f, p_gp = 0.f, p_d2 = 0.f, p_hp = 0.f, p_d3 = 0.f;
    for (int n = K - 1; n >= 0; --n) {
      const float4 c0 = __ldg(c + 3 * n);
      const float4 c1 = __ldg(c + 3 * n + 1);
      p_m1 = fmaf(p_m1, a, c0.x);
      p_g = fmaf(p_g, a, c0.y);
      p_m2 = fmaf(p_m2, a, c0.z);
      p_h = fmaf(p_h, a, c0.w);
      p_m3 = fmaf(p_m3, a, c1.x);
      if (JAC) {
        const float4 c2 = __ldg(c + 3 * n + 2);
        p_d1 = fmaf(p_d1, a, c1.y);
        p_gp = fmaf(p_gp, a, c1.z);
        p_d2 = fmaf(p_d2, a, c1.w);
        p_hp = fmaf(p_hp, a, c2.x);
        p_d3 = fmaf(p_d3, a, c2.y);
      }
    }
    const float E = expf(-y);
    const float G = E * p_g, H = E * p_h;
    const float A = fmaf(I, G, E * p_m2);
    const float B = fmaf(Jr, D, fmaf(I, H, E * p_m3));
    const int code = __ldg(kd.iv_code + iv);
    if (JAC) {
      const float Gp = -E * p_gp, Hp = -E * p_hp;
      const float Ap = fmaf(Ip, G, fmaf(I, Gp, -E * p_d2));
      const float Bp = fmaf(Jp, D, fmaf(Ip, H, fmaf(I, Hp, -E * p_d3)));
      Ip = fmaf(E, fmaf(-D, I, Ip), -E * p_d1);
      Jp += Ap;
      if (code >= 0) {   // gaps between frames propagate the state only
        SAp += Ap;
        SBp += Bp;
      }
    }
    I = fmaf(E, I, E * p_m1);
    Jr += A;
    if (code >= 0) {
      SA += A;
      SB += B;
    }
    if (code >= 0 && (code & 1)) {
      const int m = code >> 1;
      const float inv = __ldg(kd.fr_inv + m);
      const float cp = __ldg(kd.fr_cp + m);
      const float S = fmaf(k3, SB, SA) * inv;   // frame average of C_T / K1
      const float T = K1 * S;
      const float F = fmaf(Vb, cp - T, T);      // (1 - Vb) T + Vb cp
      if (JAC) {
        // dC_T/dk2 = K1 (dI/da + k3 dJ/da); dC_T/dk3 = K1 (dI/da + J + k3 dJ/da),
        // and dI/da + J = -a dJ/da (from I' = Cp - a I), so dC_T/dk3 = -K1 k2 dJ/da:
        // a single non-negative term, exactly 0 at k2 = 0 instead of a cancelling
        // difference.
        const float w = 1.f - Vb;
        const float Sp = fmaf(k3, SBp, SAp) * inv;
        sink(m, F, w * S, w * K1 * Sp, -w * K1 * k2 * SBp * inv, cp - T);
      } else {
        sink(m, F, 0.f, 0.f, 0.f, 0.f);
      }
      SA = SB = SAp = SBp = 0.f;
    }
  }
}

// ---------------------------------------------------------------- tac_eval
constexpr int TAC_THREADS = 128;

struct TacSink {
  float* sF;   // shared row of this voxel: M floats
  float* sJ;   // shared row: 4M floats, or null
  __device__ void operator()(int m, float F, float j0, float j1, float j2, float j3) {
    sF[m] = F;
    if (sJ) {
      sJ[4 * m + 0] = j0;
      sJ[4 * m + 1] = j1;
      sJ[4 * m + 2] = j2;
      sJ[4 * m + 3] = j3;
    }
  }
};

template <bool JAC>
__global__ void __launch_bounds__(TAC_THREADS) k_tac_eval(KinDev kd, long long n_vox,
                                                          const float* __restrict__ params,
                                                          float* __restrict__ F,
                                                          float* __restrict__ J) {
  extern __shared__ float sh[];
  const int M = kd.M;
  const int ldF = M + 1, ldJ = 4 * M + 1;
  float* sF = sh;
  float* sJ = sh + TAC_THREADS * ldF;
  const long long v0 = (long long)blockIdx.x * TAC_THREADS;
  const long long v = v0 + threadIdx.x;
  const long long nv = min((long long)TAC_THREADS, n_vox - v0);
  if (v < n_vox) {
    const float K1 = params[v], k2 = params[n_vox + v], k3 = params[2 * n_vox + v],
                Vb = params[3 * n_vox + v];
    TacSink sink{sF + threadIdx.x * ldF, JAC ? sJ + threadIdx.x * ldJ : nullptr};
    eval_model<JAC>(kd, K1, k2, k3, Vb, sink);
  }
  __syncthreads();
  for (long long e = threadIdx.x; e < nv * M; e += TAC_THREADS) {
    const long long r = e / M, m = e - r * M;
    F[v0 * M + e] = sF[r * ldF + m];
  }
  if (JAC) {
    for (long long e = threadIdx.x; e < nv * 4 * M; e += TAC_THREADS) {
      const long long r = e / (4 * M), m = e - r * 4 * M;
      J[v0 * 4 * M + e] = sJ[r * ldJ + m];
    }
  }
}

int launch_tac_eval(const kcs_kinetics* k, int64_t n_vox, const float* params, float* F, float* J,
                    cudaStream_t s) {
  if (n_vox == 0) return KCS_OK;
  const int M = k->M;
  const unsigned blocks = (unsigned)((n_vox + TAC_THREADS - 1) / TAC_THREADS);
  if (J) {
    const size_t smem = sizeof(float) * TAC_THREADS * ((M + 1) + (4 * M + 1));
    KCS_CUDA(cudaFuncSetAttribute(k_tac_eval<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    k_tac_eval<true><<<blocks, TAC_THREADS, smem, s>>>(k->dev(), n_vox, params, F, J);
  } else {
    const size_t smem = sizeof(float) * TAC_THREADS * (M + 1);
    k_tac_eval<false><<<blocks, TAC_THREADS, smem, s>>>(k->dev(), n_vox, params, F, nullptr);
  }
  KCS_LAUNCHED();
  return KCS_OK;
}

// ---------------------------------------------------------------- Ki
__global__ void k_ki(long long n, const float* p, float* ki) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const float K1 = p[v], k2 = p[n + v], k3 = p[2 * n + v];
  const float a = k2 + k3;
  ki[v] = a > 0.f ? K1 * k3 / a : 0.f;
}

// ---------------------------------------------------------------- Huber
__device__ __forceinline__ float huber_psi(float t, float d) { return fminf(fmaxf(t, -d), d); }
__device__ __forceinline__ float huber_h(float t, float d) {
  const float at = fabsf(t);
  return at <= d ? 0.5f * t * t : fmaf(d, at, -0.5f * d * d);
}

__global__ void k_huber_grad(int nx, int ny, int nz, const float* p, float delta, float* g) {
  const long long n = (long long)nx * ny * nz;
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int i = (int)(v % nx);
  const int j = (int)((v / nx) % ny);
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int dy = -1; dy <= 1; ++dy)
    for (int dx = -1; dx <= 1; ++dx) {
      if (!dx && !dy) continue;
      const int ii = i + dx, jj = j + dy;
      if (ii < 0 || ii >= nx || jj < 0 || jj >= ny) continue;
      const long long u = v + (long long)dy * nx + dx;
      for (int q = 0; q < 4; ++q) acc[q] += huber_psi(p[q * n + v] - p[q * n + u], delta);
    }
  for (int q = 0; q < 4; ++q) g[q * n + v] = acc[q];
}

// ---------------------------------------------------------------- MAP-LM
constexpr int LM_THREADS = 128;
__constant__ float c_lo[4] = {0.f, 0.f, 0.f, 0.f};
__constant__ float c_hi[4] = {2.f, 2.f, 1.f, 1.f};
constexpr float LAMBDA0 = 1e-2f, LAMBDA_MIN = 1e-7f, LAMBDA_MAX = 1e7f;
// A trial is accepted when it lowers the voxel objective by more than TAU of its
// value: smaller changes are below float32 resolution of the model.
constexpr float TAU = 1e-5f;

struct LmArgs {
  KinDev kd;
  int nx, ny, nz;
  const float* x;        // [V][M]
  const float* p_in;     // [4][V]
  float* p_out;          // [4][V]
  float* lambda;         // [V]
  int reset_lambda;
  float beta, delta;
};

struct NormalSink {
  const float* xs;   // this voxel's TAC in shared memory
  float* fc;         // this voxel's model TAC at the current point (shared memory)
  float rr;          // sum of squared residuals at the current point
  float A00, A01, A02, A03, A11, A12, A13, A22, A23, A33;
  float b0, b1, b2, b3;
  __device__ void operator()(int m, float F, float j0, float j1, float j2, float j3) {
    const float r = xs[m] - F;
    fc[m] = F;
    rr = fmaf(r, r, rr);
    A00 = fmaf(j0, j0, A00); A01 = fmaf(j0, j1, A01); A02 = fmaf(j0, j2, A02); A03 = fmaf(j0, j3, A03);
    A11 = fmaf(j1, j1, A11); A12 = fmaf(j1, j2, A12); A13 = fmaf(j1, j3, A13);
    A22 = fmaf(j2, j2, A22); A23 = fmaf(j2, j3, A23);
    A33 = fmaf(j3, j3, A33);
    b0 = fmaf(j0, r, b0); b1 = fmaf(j1, r, b1); b2 = fmaf(j2, r, b2); b3 = fmaf(j3, r, b3);
  }
};

// Change of the data term between the current point (fc) and the trial,
// 1/2 sum (x - F')^2 - 1/2 sum (x - F)^2 = sum (F - F') (x - (F + F')/2),
// accumulated directly so that small decreases are not lost in the rounding of
// two large sums.
struct DeltaSink {
  const float* xs;
  const float* fc;
  float dphi;
  __device__ void operator()(int m, float F, float, float, float, float) {
    const float Fc = fc[m];
    dphi = fmaf(Fc - F, xs[m] - 0.5f * (Fc + F), dphi);
  }
};

// Cholesky solve of the damped 4x4 normal equations in float64.  Returns
// false (no step) if a pivot is not positive.
__device__ bool solve4(const NormalSink& s, double lam, const double rhs[4], double out[4]) {
  const double A00 = (double)s.A00 + lam, A11 = (double)s.A11 + lam, A22 = (double)s.A22 + lam,
               A33 = (double)s.A33 + lam;
  const double A10 = s.A01, A20 = s.A02, A30 = s.A03, A21 = s.A12, A31 = s.A13, A32 = s.A23;
  if (!(A00 > 0.0)) return false;
  const double i0 = rsqrt(A00);
  const double L10 = A10 * i0, L20 = A20 * i0, L30 = A30 * i0;
  const double d1 = A11 - L10 * L10;
  if (!(d1 > 0.0)) return false;
  const double i1 = rsqrt(d1);
  const double L21 = (A21 - L20 * L10) * i1, L31 = (A31 - L30 * L10) * i1;
  const double d2 = A22 - L20 * L20 - L21 * L21;
  if (!(d2 > 0.0)) return false;
  const double i2 = rsqrt(d2);
  const double L32 = (A32 - L30 * L20 - L31 * L21) * i2;
  const double d3 = A33 - L30 * L30 - L31 * L31 - L32 * L32;
  if (!(d3 > 0.0)) return false;
  const double i3 = rsqrt(d3);
  const double z0 = rhs[0] * i0;
  const double z1 = (rhs[1] - L10 * z0) * i1;
  const double z2 = (rhs[2] - L20 * z0 - L21 * z1) * i2;
  const double z3 = (rhs[3] - L30 * z0 - L31 * z1 - L32 * z2) * i3;
  out[3] = z3 * i3;
  out[2] = (z2 - L32 * out[3]) * i2;
  out[1] = (z1 - L21 * out[2] - L31 * out[3]) * i1;
  out[0] = (z0 - L10 * out[1] - L20 * out[2] - L30 * out[3]) * i0;
  return true;
}

__global__ void __launch_bounds__(LM_THREADS) k_lm_step(LmArgs L) {
  extern __shared__ float xs_all[];
  const int M = L.kd.M;
  const int ld = M + 1;
  float* fc_all = xs_all + LM_THREADS * ld;
  const long long V = (long long)L.nx * L.ny * L.nz;
  const long long v0 = (long long)blockIdx.x * LM_THREADS;
  const long long v = v0 + threadIdx.x;
  const long long nv = min((long long)LM_THREADS, V - v0);
  for (long long e = threadIdx.x; e < nv * M; e += LM_THREADS) {
    const long long r = e / M, m = e - r * M;
    xs_all[r * ld + m] = L.x[v0 * M + e];
  }
  __syncthreads();
  if (v >= V) return;
  const float* xs = xs_all + threadIdx.x * ld;
  const int i = (int)(v % L.nx);
  const int j = (int)((v / L.nx) % L.ny);
  float xi[4];
  for (int q = 0; q < 4; ++q) xi[q] = L.p_in[q * V + v];
  // Huber gradient and potential at the current point (neighbours frozen).
  float g[4] = {0.f, 0.f, 0.f, 0.f};
  float Hc = 0.f;
  for (int dy = -1; dy <= 1; ++dy)
    for (int dx = -1; dx <= 1; ++dx) {
      if (!dx && !dy) continue;
      const int ii = i + dx, jj = j + dy;
      if (ii < 0 || ii >= L.nx || jj < 0 || jj >= L.ny) continue;
      const long long u = v + (long long)dy * L.nx + dx;
      for (int q = 0; q < 4; ++q) {
        const float t = xi[q] - L.p_in[q * V + u];
        g[q] += huber_psi(t, L.delta);
        Hc += huber_h(t, L.delta);
      }
    }
  float* fc = fc_all + threadIdx.x * ld;
  NormalSink ns{xs, fc, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  eval_model<true>(L.kd, xi[0], xi[1], xi[2], xi[3], ns);
  float lam = L.reset_lambda ? LAMBDA0 : L.lambda[v];
  const double rhs[4] = {(double)ns.b0 - (double)L.beta * g[0], (double)ns.b1 - (double)L.beta * g[1],
                         (double)ns.b2 - (double)L.beta * g[2], (double)ns.b3 - (double)L.beta * g[3]};
  double step[4];
  bool accept = false;
  float tr[4];
  if (solve4(ns, (double)lam, rhs, step)) {
    for (int q = 0; q < 4; ++q) tr[q] = fminf(fmaxf(xi[q] + (float)step[q], c_lo[q]), c_hi[q]);
    DeltaSink ds{xs, fc, 0.f};
    eval_model<false>(L.kd, tr[0], tr[1], tr[2], tr[3], ds);
    float dH = 0.f;   // H(trial) - H(current), neighbours frozen
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        if (!dx && !dy) continue;
        const int ii = i + dx, jj = j + dy;
        if (ii < 0 || ii >= L.nx || jj < 0 || jj >= L.ny) continue;
        const long long u = v + (long long)dy * L.nx + dx;
        for (int q = 0; q < 4; ++q) {
          const float nb = L.p_in[q * V + u];
          dH += huber_h(tr[q] - nb, L.delta) - huber_h(xi[q] - nb, L.delta);
        }
      }
    // Phi(trial) - Phi(current) < -TAU Phi(current)
    const float phi = fmaf(0.5f, ns.rr, L.beta * Hc);
    accept = fmaf(L.beta, dH, ds.dphi) < -TAU * phi;
  }
  if (accept) {
    for (int q = 0; q < 4; ++q) L.p_out[q * V + v] = tr[q];
    lam = fmaxf(lam * 0.1f, LAMBDA_MIN);
  } else {
    for (int q = 0; q < 4; ++q) L.p_out[q * V + v] = xi[q];
    lam = fminf(lam * 10.f, LAMBDA_MAX);
  }
  L.lambda[v] = lam;
}

}  // namespace kcs

using namespace kcs;

// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n.
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

extern "C" {

int kcs_create_kinetics(kcs_kinetics_t** out, int n_frames, const double* t_start,
                        const double* t_end, const double* feng, void* stream) {
  clear_error();
  KCS_REQUIRE(out && t_start && t_end && feng, "NULL argument");
  KCS_REQUIRE(n_frames >= 4 && n_frames <= 32 && n_frames % 4 == 0,
              "n_frames=%d must be a multiple of 4 in [4, 32]", n_frames);
  std::vector<double> t0, dt, fdt(n_frames);
  std::vector<int> code;
  double t = 0.0;
  for (int m = 0; m < n_frames; ++m) {
    KCS_REQUIRE(t_end[m] > t_start[m], "frame %d has non-positive duration", m);
    KCS_REQUIRE(t_start[m] >= t - 1e-12, "frame %d starts before the previous frame ends", m);
    KCS_REQUIRE(t_start[m] >= 0.0, "frame %d starts before injection (t < 0)", m);
    if (t_start[m] > t) {   // gap: propagate without output
      const int np = (int)ceil((t_start[m] - t) / DT_MAX);
      for (int k = 0; k < np; ++k) {
        t0.push_back(t + (t_start[m] - t) * k / np);
        dt.push_back((t_start[m] - t) / np);
        code.push_back(-1);
      }
    }
    const double d = t_end[m] - t_start[m];
    const int np = (int)ceil(d / DT_MAX);
    for (int k = 0; k < np; ++k) {
      t0.push_back(t_start[m] + d * k / np);
      dt.push_back(d / np);
      code.push_back(2 * m + (k == np - 1 ? 1 : 0));
    }
    fdt[m] = d;
    t = t_end[m];
  }
  const int n_iv = (int)t0.size();
  kcs_kinetics* k = new kcs_kinetics();
  k->M = n_frames;
  k->n_iv = n_iv;
  cudaGetDevice(&k->device);
  std::vector<double> gx, gw;
  const int NGL = 16, NPANEL = 16;
  gauss_legendre(NGL, gx, gw);
  cudaStream_t s = as_stream(stream);
  const size_t nd = 2 * (size_t)n_iv + 2 * NGL + n_frames + n_iv;
  bool ok = cudaMalloc(&k->d_coef, sizeof(float) * (size_t)n_iv * KMAX * NCH) == cudaSuccess;
  ok = ok && cudaMalloc(&k->d_iv_dt, sizeof(float) * n_iv) == cudaSuccess;
  ok = ok && cudaMalloc(&k->d_iv_code, sizeof(int) * n_iv) == cudaSuccess;
  ok = ok && cudaMalloc(&k->d_fr_cp, sizeof(float) * n_frames) == cudaSuccess;
  ok = ok && cudaMalloc(&k->d_fr_inv, sizeof(float) * n_frames) == cudaSuccess;
  ok = ok && cudaMalloc(&k->d_tmp, sizeof(double) * nd) == cudaSuccess;
  if (!ok) {
    set_error("cudaMalloc failed for kinetics tables");
    kcs_destroy_kinetics(k);
    return KCS_ERR_OOM;
  }
  std::vector<double> host(nd);
  std::copy(t0.begin(), t0.end(), host.begin());
  std::copy(dt.begin(), dt.end(), host.begin() + n_iv);
  std::copy(gx.begin(), gx.end(), host.begin() + 2 * n_iv);
  std::copy(gw.begin(), gw.end(), host.begin() + 2 * n_iv + NGL);
  std::copy(fdt.begin(), fdt.end(), host.begin() + 2 * n_iv + 2 * NGL);
  std::vector<float> dtf(dt.begin(), dt.end());
  KCS_CUDA(cudaMemcpyAsync(k->d_tmp, host.data(), sizeof(double) * nd, cudaMemcpyHostToDevice, s));
  KCS_CUDA(cudaMemcpyAsync(k->d_iv_dt, dtf.data(), sizeof(float) * n_iv, cudaMemcpyHostToDevice, s));
  KCS_CUDA(cudaMemcpyAsync(k->d_iv_code, code.data(), sizeof(int) * n_iv, cudaMemcpyHostToDevice, s));
  TabArgs ta;
  ta.iv_t0 = k->d_tmp;
  ta.iv_dt = k->d_tmp + n_iv;
  ta.gl_x = k->d_tmp + 2 * n_iv;
  ta.gl_w = k->d_tmp + 2 * n_iv + NGL;
  ta.n_gl = NGL;
  ta.n_panel = NPANEL;
  ta.A1 = feng[0]; ta.A2 = feng[1]; ta.A3 = feng[2];
  ta.l1 = feng[3]; ta.l2 = feng[4]; ta.l3 = feng[5];
  ta.coef = reinterpret_cast<float*>(k->d_coef);
  ta.m0 = k->d_tmp + 2 * n_iv + 2 * NGL + n_frames;
  k_tabulate<<<n_iv, KMAX, 0, s>>>(ta);
  KCS_LAUNCHED();
  k_frame_tables<<<1, 32, 0, s>>>(ta.m0, k->d_iv_code, n_iv, k->d_tmp + 2 * n_iv + 2 * NGL,
                                  n_frames, k->d_fr_cp, k->d_fr_inv);
  KCS_LAUNCHED();
  // the host staging vectors die here: wait for the copies
  KCS_CUDA(cudaStreamSynchronize(s));
  *out = k;
  return KCS_OK;
}

int kcs_destroy_kinetics(kcs_kinetics_t* k) {
  clear_error();
  if (!k) return KCS_OK;
  cudaFree(k->d_coef);
  cudaFree(k->d_iv_dt);
  cudaFree(k->d_iv_code);
  cudaFree(k->d_fr_cp);
  cudaFree(k->d_fr_inv);
  cudaFree(k->d_tmp);
  delete k;
  return KCS_OK;
}

int kcs_tac_eval(const kcs_kinetics_t* k, int64_t n_vox, const float* params, float* F, float* J,
                 void* stream) {
  clear_error();
  KCS_REQUIRE(k && params && F, "NULL argument");
  KCS_REQUIRE(n_vox >= 0, "n_vox < 0");
  return launch_tac_eval(k, n_vox, params, F, J, as_stream(stream));
}

int kcs_ki(int64_t n_vox, const float* params, float* ki, void* stream) {
  clear_error();
  KCS_REQUIRE(params && ki, "NULL argument");
  KCS_REQUIRE(n_vox >= 0, "n_vox < 0");
  if (n_vox == 0) return KCS_OK;
  k_ki<<<(unsigned)((n_vox + 255) / 256), 256, 0, as_stream(stream)>>>(n_vox, params, ki);
  KCS_LAUNCHED();
  return KCS_OK;
}

int kcs_huber_grad(int nx, int ny, int nz, const float* params, float delta, float* grad,
                   void* stream) {
  clear_error();
  KCS_REQUIRE(params && grad, "NULL argument");
  KCS_REQUIRE(nx > 0 && ny > 0 && nz > 0, "sizes must be positive");
  KCS_REQUIRE(delta > 0.f, "delta must be positive");
  const long long n = (long long)nx * ny * nz;
  k_huber_grad<<<(unsigned)((n + 255) / 256), 256, 0, as_stream(stream)>>>(nx, ny, nz, params,
                                                                            delta, grad);
  KCS_LAUNCHED();
  return KCS_OK;
}

size_t kcs_lm_workspace_size(int nx, int ny, int nz) {
  if (nx <= 0 || ny <= 0 || nz <= 0) return 0;
  const size_t V = (size_t)nx * ny * nz;
  return align256(4 * V * sizeof(float)) + align256(V * sizeof(float));
}

int kcs_map_lm_fit(const kcs_kinetics_t* k, int nx, int ny, int nz, const float* x, float* params,
                   float* lambda, int n_steps, float beta_h, float delta, float* F_out,
                   void* workspace, size_t ws_bytes, void* stream) {
  clear_error();
  KCS_REQUIRE(k && x && params, "NULL argument");
  KCS_REQUIRE(nx > 0 && ny > 0 && nz > 0, "sizes must be positive");
  KCS_REQUIRE(n_steps >= 0, "n_steps < 0");
  KCS_REQUIRE(delta > 0.f && beta_h >= 0.f, "need delta > 0 and beta_h >= 0");
  KCS_REQUIRE(workspace && ws_bytes >= kcs_lm_workspace_size(nx, ny, nz),
              "workspace too small (%zu < %zu)", ws_bytes, kcs_lm_workspace_size(nx, ny, nz));
  cudaStream_t s = as_stream(stream);
  const long long V = (long long)nx * ny * nz;
  float* pong = static_cast<float*>(workspace);
  float* lam_ws = reinterpret_cast<float*>(static_cast<char*>(workspace) +
                                           align256(4 * (size_t)V * sizeof(float)));
  LmArgs L;
  L.kd = k->dev();
  L.nx = nx; L.ny = ny; L.nz = nz;
  L.x = x;
  L.lambda = lambda ? lambda : lam_ws;
  L.beta = beta_h;
  L.delta = delta;
  const size_t smem = sizeof(float) * LM_THREADS * (k->M + 1) * 2;
  const unsigned blocks = (unsigned)((V + LM_THREADS - 1) / LM_THREADS);
  float* cur = params;
  float* nxt = pong;
  for (int it = 0; it < n_steps; ++it) {
    L.p_in = cur;
    L.p_out = nxt;
    L.reset_lambda = (it == 0 && !lambda) ? 1 : 0;
    k_lm_step<<<blocks, LM_THREADS, smem, s>>>(L);
    KCS_LAUNCHED();
    std::swap(cur, nxt);
  }
  if (cur != params)
    KCS_CUDA(cudaMemcpyAsync(params, cur, 4 * (size_t)V * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (F_out) return launch_tac_eval(k, V, params, F_out, nullptr, s);
  return KCS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- no-allocation MAP-LM
// kcs_map_lm_fit_static: the MAP-LM fit with its scratch (ping-pong maps and
// lambda) in a fixed device array owned by this library, for callers that may
// not allocate device memory themselves.  The array lives in every GPU that
// loads the library until the process exits.
namespace {
constexpr size_t kStaticLmBytes =
    ((4 * (size_t)KCS_LM_STATIC_MAX_VOXELS * sizeof(float) + 255) & ~size_t(255)) +
    (size_t)KCS_LM_STATIC_MAX_VOXELS * sizeof(float);
static __device__ __align__(256) unsigned char g_lm_scratch[kStaticLmBytes];
constexpr int kMaxDevices = 64;
std::mutex g_lm_scratch_mu;
void* g_lm_scratch_dev[kMaxDevices] = {};   // device address of g_lm_scratch, per device
}  // namespace

extern "C" int kcs_map_lm_fit_static(const kcs_kinetics_t* k, int nx, int ny, int nz,
                                     const float* x, float* params, float* lambda, int n_steps,
                                     float beta_h, float delta, float* F_out, void* stream) {
  clear_error();
  KCS_REQUIRE(nx > 0 && ny > 0 && nz > 0, "sizes must be positive");
  const long long V = (long long)nx * ny * nz;
  KCS_REQUIRE(V <= KCS_LM_STATIC_MAX_VOXELS,
              "kcs_map_lm_fit_static handles at most %d voxels (got %lld); use kcs_map_lm_fit "
              "with a caller workspace", KCS_LM_STATIC_MAX_VOXELS, V);
  KCS_REQUIRE(kcs_lm_workspace_size(nx, ny, nz) <= kStaticLmBytes, "static scratch too small");
  int dev = 0;
  KCS_CUDA(cudaGetDevice(&dev));
  KCS_REQUIRE(dev >= 0 && dev < kMaxDevices, "device index %d out of range", dev);
  void* scratch = nullptr;
  {
    // First call on this device: look up the array's device address with the
    // device current (host code cannot use the symbol itself as a pointer).
    std::lock_guard<std::mutex> lock(g_lm_scratch_mu);
    if (!g_lm_scratch_dev[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_lm_scratch);
      if (e != cudaSuccess || !p) {
        set_error("cudaGetSymbolAddress of the static LM scratch failed: %s",
                  cudaGetErrorString(e));
        return KCS_ERR_CUDA;
      }
      g_lm_scratch_dev[dev] = p;
    }
    scratch = g_lm_scratch_dev[dev];
  }
  return kcs_map_lm_fit(k, nx, ny, nz, x, params, lambda, n_steps, beta_h, delta, F_out, scratch,
                        kStaticLmBytes, stream);
}
