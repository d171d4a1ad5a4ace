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
// float64 by Gauss-Legendre quadrature.  Given a, the frame averages A_m(a)
// (of I) and B_m(a) (of J) fix the whole model, which is linear in K1, k3 and
// Vb:  F_m = (1 - Vb) K1 (A_m + k3 B_m) + Vb cp_m.  So A_m, B_m and their
// a-derivatives are computed once, in float64, on a grid of a (spacing 1/512,
// 0 <= a <= 3.75) by running the interval recursion at every node; a voxel
// evaluates cubic Hermite interpolants of them (values and derivatives at the
// two neighbouring nodes) in float32.  Interpolation error, measured against
// the exact model: below 1.1e-8 of each frame's range for F and dF/da on the
// paper's and the configs' schedules.

#include <cmath>
#include <algorithm>
#include <type_traits>
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
  double* base;          // [n_iv][NB][10]
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
  if (n >= NB) return;
  const double D = a.iv_dt[iv];
  const double t0 = a.iv_t0[iv];
  double P[NB + 4], Q[NB + 4];   // u^j/j!, v^k/k!
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
  double* o = a.base + ((size_t)iv * NB + n) * 10;
  o[CH_M1] = m1;
  o[CH_G] = f1;
  o[CH_M2] = m2;
  o[CH_H] = f2 * (n + 1);
  o[CH_M3] = m3;
  o[CH_D1] = d1;
  o[CH_GP] = f2;
  o[CH_D2] = d2;
  o[CH_HP] = f3 * (n + 1);
  o[CH_D3] = d3;
  if (n == 0) a.m0[iv] = s0;
}

// The frame averages A_m(a), B_m(a) and their a-derivatives, in float64: per
// interval of length D the channel series sum_n a^n c_n (Horner over the NB
// base terms) and e^{-aD} advance the running integrals I(t) = int Cp
// e^{-a(t-s)} ds and J(t) = int I (and their a-derivatives, from the
// derivative channels) across the interval; the interval integrals of I and J
// are summed over each frame and divided by its duration, then handed to
// out(m, A, A', B, B').
template <class Out>
__device__ void frame_averages(double a, const double* base, const double* iv_dt,
                               const int* iv_code, int n_iv, const double* fdt, Out out) {
  double I = 0.0, Ip = 0.0, Jr = 0.0, Jp = 0.0, SA = 0.0, SB = 0.0, SAp = 0.0, SBp = 0.0;
  for (int iv = 0; iv < n_iv; ++iv) {
    const double D = iv_dt[iv];
    const double* b = base + (size_t)iv * NB * 10;
    double ch[10];
    for (int c = 0; c < 10; ++c) ch[c] = 0.0;
    for (int k = NB - 1; k >= 0; --k)
      for (int c = 0; c < 10; ++c) ch[c] = fma(ch[c], a, b[(size_t)k * 10 + c]);
    const double E = exp(-a * D);
    const double G = E * ch[CH_G], H = E * ch[CH_H];
    const double Gp = -E * ch[CH_GP], Hp = -E * ch[CH_HP];
    // interval integrals of I and J (A, B) and their a-derivatives (Ap, Bp)
    const double A = I * G + E * ch[CH_M2];
    const double B = Jr * D + I * H + E * ch[CH_M3];
    const double Ap = Ip * G + I * Gp - E * ch[CH_D2];
    const double Bp = Jp * D + Ip * H + I * Hp - E * ch[CH_D3];
    // state at the end of the interval
    Ip = E * (Ip - D * I) - E * ch[CH_D1];
    Jp += Ap;
    I = E * I + E * ch[CH_M1];
    Jr += A;
    const int code = iv_code[iv];
    if (code < 0) continue;                      // gaps propagate the state only
    SA += A;
    SB += B;
    SAp += Ap;
    SBp += Bp;
    if (code & 1) {                              // last interval of frame m
      const int m = code >> 1;
      const double inv = 1.0 / fdt[m];
      out(m, SA * inv, SAp * inv, SB * inv, SBp * inv);
      SA = SB = SAp = SBp = 0.0;
    }
  }
}

// Float64 node values (A, A', B, B') at a = n / NODES_PER_UNIT, [frame][node][4].
// One thread per node.
__global__ void k_node_table(const double* base, const double* iv_dt, const int* iv_code,
                             int n_iv, const double* fdt, int nn, double* node) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const double a = (double)n / NODES_PER_UNIT;
  frame_averages(a, base, iv_dt, iv_code, n_iv, fdt,
                 [&](int m, double A, double Ap, double B, double Bp) {
                   double* o = node + ((size_t)m * nn + n) * 4;
                   o[0] = A; o[1] = Ap; o[2] = B; o[3] = Bp;
                 });
}

// Cubic Hermite coefficients per cell and frame, in float64 from the node
// values and slopes (h = cell width): on s in [0, 1],
//   c0 = f(0), c1 = h f'(0), c2 = 3 (f(1) - f(0)) - h (2 f'(0) + f'(1)),
//   c3 = 2 (f(0) - f(1)) + h (f'(0) + f'(1)),
// then rounded once to float.  The derivative comes from the same cubic
// (c1 + 2 s c2 + 3 s^2 c3) / h: its coefficients carry the differences in
// float64, so nothing cancels in float32 (truncation ~4e-6 of the largest
// slope at h = 1/512).
__global__ void k_cell_table(const double* node, int M, int nn, float4* cell) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int nc = nn - 1;
  if (e >= M * nc) return;
  const int m = e / nc, c = e - m * nc;
  const double h = 1.0 / NODES_PER_UNIT;
  const double* n0 = node + ((size_t)m * nn + c) * 4;
  const double* n1 = n0 + 4;
  float co[2][4];
  for (int f = 0; f < 2; ++f) {
    const double f0 = n0[2 * f], d0 = n0[2 * f + 1], f1 = n1[2 * f], d1 = n1[2 * f + 1];
    co[f][0] = (float)f0;
    co[f][1] = (float)(h * d0);
    co[f][2] = (float)(3.0 * (f1 - f0) - h * (2.0 * d0 + d1));
    co[f][3] = (float)(2.0 * (f0 - f1) + h * (d0 + d1));
  }
  cell[2 * (size_t)e] = make_float4(co[0][0], co[0][1], co[0][2], co[0][3]);
  cell[2 * (size_t)e + 1] = make_float4(co[1][0], co[1][1], co[1][2], co[1][3]);
}

__global__ void k_frame_tables(const double* m0, const int* code, int n_iv, const double* fdt,
                               int M, float* fr_cp) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  double s = 0.0;
  for (int i = 0; i < n_iv; ++i)
    if (code[i] >= 0 && (code[i] >> 1) == m) s += m0[i];
  fr_cp[m] = (float)(s / fdt[m]);
}

// One table entry (the A and B cubics of a cell and frame, 32 bytes, 32-byte
// aligned) by a single 256-bit read-only load that does not allocate in L1:
// the table (M rows of cells) is served from L2, and its scattered lines would
// otherwise evict the lines that are reused (Huber neighbours).  Measured at
// full size: LM step 1.98 vs 2.12 ms, model TACs 1.37 vs 2.06 ms.
__device__ __forceinline__ void ld_cell(const float4* p, float4& a, float4& b) {
  asm("ld.global.nc.L1::no_allocate.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
      : "l"(p));
}

// ---------------------------------------------------------------- model
// Evaluates F_m (and dF_m/d(K1,k2,k3,Vb) when JAC) of VPT voxels frame by frame
// and hands each frame to sink(v, m, F, J0, J1, J2, J3).  With w = 1 - Vb and
// S = A + k3 B:  F = w K1 S + Vb cp,  dF/dK1 = w S,  dF/dk2 = w K1 (A' + k3 B'),
// dF/dk3 = w K1 (A' + B + k3 B') = -w K1 k2 B'  (A' + B = -a B' from
// I' = Cp - a I: a single term, exactly 0 at k2 = 0, instead of a cancelling
// difference),  dF/dVb = cp - K1 S.  A, B are the per-cell cubics of the
// table (cubic Hermite interpolants of the float64 node values and slopes),
// A', B' their derivatives.
template <int VPT, bool JAC, int MU = 1, class Sink>
__device__ __forceinline__ void eval_model(const KinDev& kd, const float (&K1)[VPT],
                                           const float (&k2)[VPT], const float (&k3)[VPT],
                                           const float (&Vb)[VPT], Sink& sink) {
  int j[VPT];
  float t[VPT], d2[VPT], d3[VPT];
#pragma unroll
  for (int v = 0; v < VPT; ++v) {
    const float a = fmaxf(k2[v] + k3[v], 0.f);
    const float u = a * (float)NODES_PER_UNIT;
    j[v] = min((int)u, N_CELLS - 1);                // a beyond A_MAX extrapolates
    t[v] = u - (float)j[v];
    d2[v] = 2.f * t[v];
    d3[v] = 3.f * t[v] * t[v];
  }
#pragma unroll MU
  for (int m = 0; m < kd.M; ++m) {
    const float cp = __ldg(kd.fr_cp + m);
    const float4* row = kd.cell + (size_t)m * N_CELLS * 2;
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      float4 ca, cb;
      ld_cell(row + 2 * j[v], ca, cb);
      const float A = fmaf(t[v], fmaf(t[v], fmaf(t[v], ca.w, ca.z), ca.y), ca.x);
      const float B = fmaf(t[v], fmaf(t[v], fmaf(t[v], cb.w, cb.z), cb.y), cb.x);
      const float S = fmaf(k3[v], B, A);
      const float T = K1[v] * S;
      const float F = fmaf(Vb[v], cp - T, T);       // (1 - Vb) T + Vb cp
      if (JAC) {
        // h A' and h B' (h = 1 / NODES_PER_UNIT, a power of two: exact scaling)
        const float Aph = fmaf(d3[v], ca.w, fmaf(d2[v], ca.z, ca.y));
        const float Bph = fmaf(d3[v], cb.w, fmaf(d2[v], cb.z, cb.y));
        const float w = 1.f - Vb[v];
        const float wK = w * K1[v] * (float)NODES_PER_UNIT;
        sink(v, m, F, w * S, wK * fmaf(k3[v], Bph, Aph), -wK * k2[v] * Bph, cp - T);
      } else {
        sink(v, m, F, 0.f, 0.f, 0.f, 0.f);
      }
    }
  }
}

// ---------------------------------------------------------------- tac_eval
constexpr int TAC_THREADS = 128;
// frames per trip of the model loop in k_tac_eval (one voxel per thread: two
// frames' table reads in flight)
#ifndef KCS_TAC_UNROLL
#define KCS_TAC_UNROLL 2
#endif

struct TacSink {
  float* sF;   // shared row of this voxel: M floats
  float* sJ;   // shared row: 4M floats, or null
  __device__ void operator()(int, int m, float F, float j0, float j1, float j2, float j3) {
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
    const float K1[1] = {params[v]}, k2[1] = {params[n_vox + v]}, k3[1] = {params[2 * n_vox + v]},
                Vb[1] = {params[3 * n_vox + v]};
    TacSink sink{sF + threadIdx.x * ldF, JAC ? sJ + threadIdx.x * ldJ : nullptr};
    eval_model<1, JAC, KCS_TAC_UNROLL>(kd, K1, k2, k3, Vb, sink);
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

// ---------------------------------------------------------------- tac_vjp
// gparams[q][v] = sum_m dF_vm/dxi_q gF_vm: the kinetic Jacobian transposed,
// applied to a gradient with respect to the model TACs (reverse mode of
// kcs_tac_eval).
struct VjpSink {
  const float* g;   // this voxel's gF row in shared memory
  float acc[4];
  __device__ void operator()(int, int m, float, float j0, float j1, float j2, float j3) {
    const float gm = g[m];
    acc[0] = fmaf(j0, gm, acc[0]);
    acc[1] = fmaf(j1, gm, acc[1]);
    acc[2] = fmaf(j2, gm, acc[2]);
    acc[3] = fmaf(j3, gm, acc[3]);
  }
};

__global__ void __launch_bounds__(TAC_THREADS) k_tac_vjp(KinDev kd, long long n_vox,
                                                         const float* __restrict__ params,
                                                         const float* __restrict__ gF,
                                                         float* __restrict__ gparams) {
  extern __shared__ float sg[];
  const int M = kd.M;
  const int ld = M + 1;
  const long long v0 = (long long)blockIdx.x * TAC_THREADS;
  const long long v = v0 + threadIdx.x;
  const long long nv = min((long long)TAC_THREADS, n_vox - v0);
  for (int e = threadIdx.x; e < (int)nv * M; e += TAC_THREADS) {
    const int r = (int)__umulhi((unsigned)e, kd.div_m), m = e - r * M;
    sg[r * ld + m] = gF[v0 * M + e];
  }
  __syncthreads();
  if (v >= n_vox) return;
  const float K1[1] = {params[v]}, k2[1] = {params[n_vox + v]}, k3[1] = {params[2 * n_vox + v]},
              Vb[1] = {params[3 * n_vox + v]};
  VjpSink sink{sg + threadIdx.x * ld, {0.f, 0.f, 0.f, 0.f}};
  eval_model<1, true>(kd, K1, k2, k3, Vb, sink);
#pragma unroll
  for (int q = 0; q < 4; ++q) gparams[q * n_vox + v] = sink.acc[q];
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

// nb3d = 0: the 8 in-plane neighbours (Sec. II-C); 1: the 26 of the 3x3x3 cube.
__global__ void k_huber_grad(int nx, int ny, int nz, const float* p, float delta, int nb3d,
                             float* g) {
  const long long n = (long long)nx * ny * nz;
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int i = (int)(v % nx);
  const int j = (int)((v / nx) % ny);
  const int k = (int)(v / ((long long)nx * ny));
  const int dz0 = nb3d ? -1 : 0, dz1 = nb3d ? 1 : 0;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int dz = dz0; dz <= dz1; ++dz) {
    const int kk = k + dz;
    if (kk < 0 || kk >= nz) continue;
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        if (!dx && !dy && !dz) continue;
        const int ii = i + dx, jj = j + dy;
        if (ii < 0 || ii >= nx || jj < 0 || jj >= ny) continue;
        const long long u = v + ((long long)dz * ny + dy) * nx + dx;
        for (int q = 0; q < 4; ++q) acc[q] += huber_psi(p[q * n + v] - p[q * n + u], delta);
      }
  }
  for (int q = 0; q < 4; ++q) g[q * n + v] = acc[q];
}

// ---------------------------------------------------------------- MAP-LM
#ifndef KCS_LM_VPT
#define KCS_LM_VPT 1
#endif
#ifndef KCS_LM_CARVEOUT
#define KCS_LM_CARVEOUT 50   // percent of the maximum shared memory per SM
#endif
// frames per trip of the model loop in the LM kernels: 2, 1 % faster than 1
// now that the table reads are served from L2.  Blocks per SM: 7 (a
// 72-register budget), 1.94 vs 1.98 ms per step at 8 blocks (64 registers);
// 7 blocks with 3 or 4 frames per trip 1.97 / 1.96, 6 blocks (80 registers)
// 20 % slower, 2 voxels per thread 80 %
#ifndef KCS_LM_UNROLL
#define KCS_LM_UNROLL 2
#endif
#ifndef KCS_LM_MINBLOCKS
#define KCS_LM_MINBLOCKS 7
#endif
constexpr int LM_THREADS = 128;
constexpr int LM_VPT = KCS_LM_VPT;              // voxels per thread
constexpr int LM_BLOCK_VOX = LM_THREADS * LM_VPT;
__constant__ float c_lo[4] = {0.f, 0.f, 0.f, 0.f};
__constant__ float c_hi[4] = {2.f, 2.f, 1.f, 1.f};
constexpr float LAMBDA0 = 1e-2f, LAMBDA_MIN = 1e-7f, LAMBDA_MAX = 1e7f;

struct LmArgs {
  KinDev kd;
  int nx, ny, nz;
  const void* x;         // [V][M], storage type of the kernel instance
  const float* x_scale;  // [M] per-frame scale of a stored image (null: 1)
  const float* p_in;     // [4][V]
  float* p_out;          // [4][V]
  float* lambda;         // [V]
  int reset_lambda;
  float beta, delta;
  float tau;             // accept iff the objective falls by more than tau of its value
  int nb3d;              // Huber neighbourhood: 0 in-plane 3x3, 1 the 3x3x3 cube
  int x_al32;            // x starts on a 32-byte boundary
  const float* ne_in;    // [V][16] normal equations at the current point
  float* ne_out;         // [V][16] normal equations at the returned point
  unsigned long long div_nx, div_nxy;   // div_magic64(nx), div_magic64(nx ny)
};

// Column, row and plane of voxel v.
__device__ __forceinline__ void voxel_ijz(const LmArgs& L, long long v, int& i, int& j, int& z) {
  const unsigned long long row = div64((unsigned long long)v, L.div_nx);   // v / nx
  const unsigned long long pl = div64((unsigned long long)v, L.div_nxy);   // v / (nx ny)
  i = (int)((unsigned long long)v - row * (unsigned long long)L.nx);
  j = (int)(row - pl * (unsigned long long)L.ny);
  z = (int)pl;
}

// Compensated (Kahan) float32 sum: the value is s - c.
struct KSum {
  float s, c;
  __device__ __forceinline__ void add(float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

// Damped normal equations of one voxel, accumulated frame by frame in float32.
struct Normal {
  float A00, A01, A02, A03, A11, A12, A13, A22, A23, A33;
  float b0, b1, b2, b3;
};

struct NormalSink {
  const float* xs[LM_VPT];   // the voxels' TACs in shared memory
  Normal n[LM_VPT];
  KSum rr[LM_VPT];           // sum of squared residuals at the current point
  __device__ void operator()(int v, int m, float F, float j0, float j1, float j2, float j3) {
    const float r = xs[v][m] - F;
    rr[v].add(r * r);
    Normal& s = n[v];
    s.A00 = fmaf(j0, j0, s.A00); s.A01 = fmaf(j0, j1, s.A01); s.A02 = fmaf(j0, j2, s.A02);
    s.A03 = fmaf(j0, j3, s.A03); s.A11 = fmaf(j1, j1, s.A11); s.A12 = fmaf(j1, j2, s.A12);
    s.A13 = fmaf(j1, j3, s.A13); s.A22 = fmaf(j2, j2, s.A22); s.A23 = fmaf(j2, j3, s.A23);
    s.A33 = fmaf(j3, j3, s.A33);
    s.b0 = fmaf(j0, r, s.b0); s.b1 = fmaf(j1, r, s.b1); s.b2 = fmaf(j2, r, s.b2);
    s.b3 = fmaf(j3, r, s.b3);
  }
};


// Float-float arithmetic for the 4x4 solve: a value is hi + lo with |lo| at
// most half an ulp of hi (about 48 significant bits).  Built from the
// error-free sum (Knuth's two-sum) and product (Dekker's, here with a fused
// multiply-add).  Float64 runs at 1/64 of the float32 rate on this GPU, so the
// float-float solve costs a small fraction of the float64 one at a precision
// far beyond that of the float32-accumulated normal equations it solves.
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff ff_quick(float a, float b) {   // |a| >= |b|
  const float s = a + b;
  return ff{s, b - (s - a)};
}
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return ff{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ff ff_two_prod(float a, float b) {
  const float p = a * b;
  return ff{p, fmaf(a, b, -p)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = ff_two_sum(a.hi, b.hi);
  return ff_quick(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff{-b.hi, -b.lo}); }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const ff p = ff_two_prod(a.hi, b.hi);
  return ff_quick(p.hi, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo)));
}
__device__ __forceinline__ ff ff_mulf(ff a, float b) {
  const ff p = ff_two_prod(a.hi, b);
  return ff_quick(p.hi, fmaf(a.lo, b, p.lo));
}

// 1/sqrt(d) for 1e-30 < d < 1e30: float seed r, then one Newton step
// r <- r + r (1 - d r^2) / 2 with the residual 1 - d r^2 formed in float-float,
// which squares the seed's relative error (~1e-7 -> ~1e-14).
__device__ __forceinline__ ff ff_rsqrt(ff d) {
  const float r = rsqrtf(d.hi);
  const ff e = ff_sub(ff{1.f, 0.f}, ff_mul(d, ff_two_prod(r, r)));
  return ff_quick(r, 0.5f * r * (e.hi + e.lo));
}

// Cholesky solve of the damped 4x4 normal equations in float-float.  Returns
// false (no step) if a pivot is not positive.
__device__ bool solve4(const Normal& s, float lam, const ff rhs[4], float out[4]) {
  const ff A00 = ff_two_sum(s.A00, lam), A11 = ff_two_sum(s.A11, lam),
           A22 = ff_two_sum(s.A22, lam), A33 = ff_two_sum(s.A33, lam);
  // pivots never exceed their diagonal entry, so bounding the diagonal keeps
  // every pivot, and every square formed below, inside the float range
  if (!(A00.hi < 1e30f && A11.hi < 1e30f && A22.hi < 1e30f && A33.hi < 1e30f)) return false;
  if (!(A00.hi > 1e-30f)) return false;
  const ff i0 = ff_rsqrt(A00);
  const ff L10 = ff_mulf(i0, s.A01), L20 = ff_mulf(i0, s.A02), L30 = ff_mulf(i0, s.A03);
  const ff d1 = ff_sub(A11, ff_mul(L10, L10));
  if (!(d1.hi > 1e-30f)) return false;
  const ff i1 = ff_rsqrt(d1);
  const ff L21 = ff_mul(ff_sub(ff{s.A12, 0.f}, ff_mul(L20, L10)), i1);
  const ff L31 = ff_mul(ff_sub(ff{s.A13, 0.f}, ff_mul(L30, L10)), i1);
  const ff d2 = ff_sub(ff_sub(A22, ff_mul(L20, L20)), ff_mul(L21, L21));
  if (!(d2.hi > 1e-30f)) return false;
  const ff i2 = ff_rsqrt(d2);
  const ff L32 = ff_mul(ff_sub(ff_sub(ff{s.A23, 0.f}, ff_mul(L30, L20)), ff_mul(L31, L21)), i2);
  const ff d3 = ff_sub(ff_sub(ff_sub(A33, ff_mul(L30, L30)), ff_mul(L31, L31)), ff_mul(L32, L32));
  if (!(d3.hi > 1e-30f)) return false;
  const ff i3 = ff_rsqrt(d3);
  const ff z0 = ff_mul(rhs[0], i0);
  const ff z1 = ff_mul(ff_sub(rhs[1], ff_mul(L10, z0)), i1);
  const ff z2 = ff_mul(ff_sub(ff_sub(rhs[2], ff_mul(L20, z0)), ff_mul(L21, z1)), i2);
  const ff z3 =
      ff_mul(ff_sub(ff_sub(ff_sub(rhs[3], ff_mul(L30, z0)), ff_mul(L31, z1)), ff_mul(L32, z2)), i3);
  const ff o3 = ff_mul(z3, i3);
  const ff o2 = ff_mul(ff_sub(z2, ff_mul(L32, o3)), i2);
  const ff o1 = ff_mul(ff_sub(ff_sub(z1, ff_mul(L21, o2)), ff_mul(L31, o3)), i1);
  const ff o0 =
      ff_mul(ff_sub(ff_sub(ff_sub(z0, ff_mul(L10, o1)), ff_mul(L20, o2)), ff_mul(L30, o3)), i0);
  out[0] = o0.hi + o0.lo;
  out[1] = o1.hi + o1.lo;
  out[2] = o2.hi + o2.lo;
  out[3] = o3.hi + o3.lo;
  return true;
}

// Huber gradient of a voxel and the potential of a given point against the
// frozen neighbours.
__device__ __forceinline__ void huber_terms(const LmArgs& L, long long V, long long v, int i, int j,
                                            int k, const float (&pt)[4], float (&g)[4], float& H) {
  g[0] = g[1] = g[2] = g[3] = 0.f;
  H = 0.f;
  const int dz0 = L.nb3d ? -1 : 0, dz1 = L.nb3d ? 1 : 0;
  for (int dz = dz0; dz <= dz1; ++dz) {
    const int kk = k + dz;
    if (kk < 0 || kk >= L.nz) continue;
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        if (!dx && !dy && !dz) continue;
        const int ii = i + dx, jj = j + dy;
        if (ii < 0 || ii >= L.nx || jj < 0 || jj >= L.ny) continue;
        const long long u = v + ((long long)dz * L.ny + dy) * L.nx + dx;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float t = pt[q] - __ldg(L.p_in + q * V + u);
          g[q] += huber_psi(t, L.delta);
          H += huber_h(t, L.delta);
        }
      }
  }
}

// The damped normal equations of a voxel at its current point, kept between
// steps in the workspace as 16 contiguous floats per voxel, [V][16] (64 bytes,
// moved by two 256-bit accesses): A00 A01 A02 A03 A11 A12 A13 A22 A23 A33,
// b0..b3 (J^T r), and the compensated sum of squared residuals (s, c).
constexpr int NE_FIELDS = 16;

__device__ __forceinline__ void store_normal(float* ne, long long V, long long v, const Normal& n,
                                             const KSum& rr) {
  const float f[NE_FIELDS] = {n.A00, n.A01, n.A02, n.A03, n.A11, n.A12, n.A13, n.A22,
                              n.A23, n.A33, n.b0,  n.b1,  n.b2,  n.b3,  rr.s,  rr.c};
  float* o = ne + (size_t)v * NE_FIELDS;
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(o), "f"(f[0]),
               "f"(f[1]), "f"(f[2]), "f"(f[3]), "f"(f[4]), "f"(f[5]), "f"(f[6]), "f"(f[7]) : "memory");
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(o + 8), "f"(f[8]),
               "f"(f[9]), "f"(f[10]), "f"(f[11]), "f"(f[12]), "f"(f[13]), "f"(f[14]), "f"(f[15])
               : "memory");
}

__device__ __forceinline__ void load_normal(const float* ne, long long V, long long v, Normal& n,
                                            KSum& rr) {
  float f[NE_FIELDS];
  const float* o = ne + (size_t)v * NE_FIELDS;
  // read once per step: no L1 allocation
  asm("ld.global.nc.L1::no_allocate.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(f[0]), "=f"(f[1]), "=f"(f[2]), "=f"(f[3]), "=f"(f[4]), "=f"(f[5]), "=f"(f[6]), "=f"(f[7])
      : "l"(o));
  asm("ld.global.nc.L1::no_allocate.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(f[8]), "=f"(f[9]), "=f"(f[10]), "=f"(f[11]), "=f"(f[12]), "=f"(f[13]), "=f"(f[14]),
        "=f"(f[15])
      : "l"(o + 8));
  n = Normal{f[0], f[1], f[2], f[3], f[4], f[5], f[6], f[7], f[8], f[9], f[10], f[11], f[12], f[13]};
  rr = KSum{f[14], f[15]};
}

// Stage the block's TACs (stored type -> activity) in shared memory.
template <class TX>
__device__ __forceinline__ void stage_tacs(const LmArgs& L, float* xs_all, long long v0,
                                           long long nv) {
  const int M = L.kd.M;
  const int ld = M + 1;
  const TX* xg = static_cast<const TX*>(L.x) + v0 * M;
  if constexpr (std::is_same<TX, float>::value) {
    if (L.x_al32 && (M & 7) == 0) {
      // 8 frames of one voxel per 256-bit load (M is a multiple of 8; read
      // once into shared memory: no L1 allocation)
      for (int e8 = threadIdx.x; e8 < (int)nv * M / 8; e8 += LM_THREADS) {
        const int e = 8 * e8;
        const int r = (int)__umulhi((unsigned)e, L.kd.div_m), m = e - r * M;
        float v[8];
        asm("ld.global.nc.L1::no_allocate.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]),
              "=f"(v[7])
            : "l"(xg + e));
#pragma unroll
        for (int u = 0; u < 8; ++u)
          xs_all[r * ld + m + u] = L.x_scale ? v[u] * __ldg(L.x_scale + m + u) : v[u];
      }
      __syncthreads();
      return;
    }
  }
  if constexpr (!std::is_same<TX, float>::value) {
    if (L.x_al32 && (M & 7) == 0) {
      // 8 frames of one voxel per 16-byte load (read once: no L1 allocation),
      // converted exactly to float32
      for (int e8 = threadIdx.x; e8 < (int)nv * M / 8; e8 += LM_THREADS) {
        const int e = 8 * e8;
        const int r = (int)__umulhi((unsigned)e, L.kd.div_m), m = e - r * M;
        uint32_t w[4];
        asm("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
            : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3])
            : "l"(xg + e));
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          float2 f;
          if constexpr (std::is_same<TX, __nv_bfloat16>::value)
            f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[h]));
          else
            f = __half22float2(*reinterpret_cast<const __half2*>(&w[h]));
          const int mm = m + 2 * h;
          xs_all[r * ld + mm] = L.x_scale ? f.x * __ldg(L.x_scale + mm) : f.x;
          xs_all[r * ld + mm + 1] = L.x_scale ? f.y * __ldg(L.x_scale + mm + 1) : f.y;
        }
      }
      __syncthreads();
      return;
    }
  }
  // e < LM_BLOCK_VOX * 32: the multiply-high quotient is exact
  for (int e = threadIdx.x; e < (int)nv * M; e += LM_THREADS) {
    const int r = (int)__umulhi((unsigned)e, L.kd.div_m), m = e - r * M;
    const float xv = ld1(xg + e);
    xs_all[r * ld + m] = L.x_scale ? xv * __ldg(L.x_scale + m) : xv;
  }
  __syncthreads();
}

// Normal equations at the start maps p_in (before the first step).
template <class TX>
__global__ void __launch_bounds__(LM_THREADS, KCS_LM_MINBLOCKS) k_lm_normal(LmArgs L) {
  extern __shared__ float xs_all[];
  const int ld = L.kd.M + 1;
  const long long V = (long long)L.nx * L.ny * L.nz;
  const long long v0 = (long long)blockIdx.x * LM_BLOCK_VOX;
  const long long nv = min((long long)LM_BLOCK_VOX, V - v0);
  stage_tacs<TX>(L, xs_all, v0, nv);
  long long vv[LM_VPT];
  bool act[LM_VPT];
  float K1[LM_VPT], k2[LM_VPT], k3[LM_VPT], Vb[LM_VPT];
  NormalSink ns;
#pragma unroll
  for (int k = 0; k < LM_VPT; ++k) {
    const int lv = threadIdx.x + k * LM_THREADS;
    act[k] = lv < nv;
    vv[k] = act[k] ? v0 + lv : v0;      // inactive slots shadow a valid voxel, write nothing
    K1[k] = L.p_in[vv[k]];
    k2[k] = L.p_in[V + vv[k]];
    k3[k] = L.p_in[2 * V + vv[k]];
    Vb[k] = L.p_in[3 * V + vv[k]];
    ns.xs[k] = xs_all + (act[k] ? lv : 0) * ld;
    ns.n[k] = Normal{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    ns.rr[k] = KSum{0.f, 0.f};
  }
  eval_model<LM_VPT, true, KCS_LM_UNROLL>(L.kd, K1, k2, k3, Vb, ns);
#pragma unroll
  for (int k = 0; k < LM_VPT; ++k)
    if (act[k]) store_normal(L.ne_out, V, vv[k], ns.n[k], ns.rr[k]);
}

// One synchronous MAP-LM step.  The normal equations at the current point come
// from the workspace (written by the previous step or k_lm_normal); the model
// and its Jacobian are evaluated once, at the trial point, which yields both
// the trial objective and, if the trial is accepted, the next step's normal
// equations.  A rejected trial keeps the current ones (only lambda changes).
template <class TX>
__global__ void __launch_bounds__(LM_THREADS, KCS_LM_MINBLOCKS) k_lm_step(LmArgs L) {
  extern __shared__ float xs_all[];
  const int ld = L.kd.M + 1;
  const long long V = (long long)L.nx * L.ny * L.nz;
  const long long v0 = (long long)blockIdx.x * LM_BLOCK_VOX;
  const long long nv = min((long long)LM_BLOCK_VOX, V - v0);
  stage_tacs<TX>(L, xs_all, v0, nv);
  long long vv[LM_VPT];
  bool act[LM_VPT];
  float tr[LM_VPT][4], phi[LM_VPT], Hc[LM_VPT], lam[LM_VPT], rrs[LM_VPT], rrcmp[LM_VPT];
  bool solved[LM_VPT];
#pragma unroll
  for (int k = 0; k < LM_VPT; ++k) {
    const int lv = threadIdx.x + k * LM_THREADS;
    act[k] = lv < nv;
    const long long v = act[k] ? v0 + lv : v0;
    vv[k] = v;
    int i, j, z;
    voxel_ijz(L, v, i, j, z);
    const float xi[4] = {L.p_in[v], L.p_in[V + v], L.p_in[2 * V + v], L.p_in[3 * V + v]};
    Normal n;
    KSum rr;
    load_normal(L.ne_in, V, v, n, rr);
    rrs[k] = rr.s;
    rrcmp[k] = rr.c;
    float g[4];
    huber_terms(L, V, v, i, j, z, xi, g, Hc[k]);
    phi[k] = fmaf(0.5f, rr.s - rr.c, L.beta * Hc[k]);
    lam[k] = L.reset_lambda ? LAMBDA0 : L.lambda[v];
    const float bq[4] = {n.b0, n.b1, n.b2, n.b3};
    ff rhs[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) rhs[q] = ff_sub(ff{bq[q], 0.f}, ff_two_prod(L.beta, g[q]));
    float step[4];
    solved[k] = solve4(n, lam[k], rhs, step);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      tr[k][q] = solved[k] ? fminf(fmaxf(xi[q] + step[q], c_lo[q]), c_hi[q]) : xi[q];
  }
  NormalSink ns;
#pragma unroll
  for (int k = 0; k < LM_VPT; ++k) {
    ns.xs[k] = xs_all + (act[k] ? (int)(vv[k] - v0) : 0) * ld;
    ns.n[k] = Normal{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    ns.rr[k] = KSum{0.f, 0.f};
  }
  {
    float t1[LM_VPT], t2[LM_VPT], t3[LM_VPT], t4[LM_VPT];
#pragma unroll
    for (int k = 0; k < LM_VPT; ++k) {
      t1[k] = tr[k][0]; t2[k] = tr[k][1]; t3[k] = tr[k][2]; t4[k] = tr[k][3];
    }
    eval_model<LM_VPT, true, KCS_LM_UNROLL>(L.kd, t1, t2, t3, t4, ns);
  }
#pragma unroll
  for (int k = 0; k < LM_VPT; ++k) {
    if (!act[k]) continue;
    const long long v = vv[k];
    int i, j, z;
    voxel_ijz(L, v, i, j, z);
    float gt[4], Ht;
    huber_terms(L, V, v, i, j, z, tr[k], gt, Ht);
    // Phi(trial) - Phi(current) < -tau Phi(current)
    const float dphi = 0.5f * ((ns.rr[k].s - rrs[k]) - (ns.rr[k].c - rrcmp[k]));
    const bool accept = solved[k] && fmaf(L.beta, Ht - Hc[k], dphi) < -L.tau * phi[k];
#pragma unroll
    for (int q = 0; q < 4; ++q) L.p_out[q * V + v] = accept ? tr[k][q] : L.p_in[q * V + v];
    L.lambda[v] = accept ? fmaxf(lam[k] * 0.1f, LAMBDA_MIN) : fminf(lam[k] * 10.f, LAMBDA_MAX);
    if (accept) {
      store_normal(L.ne_out, V, v, ns.n[k], ns.rr[k]);
    } else {
      Normal nk;
      KSum rk;
      load_normal(L.ne_in, V, v, nk, rk);
      store_normal(L.ne_out, V, v, nk, rk);
    }
  }
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
  double* d_node64 = nullptr;   // float64 node values, freed once the cell table exists
  bool ok = cudaMalloc(&k->d_cell, sizeof(float4) * 2 * (size_t)n_frames * N_CELLS) == cudaSuccess;
  ok = ok && cudaMalloc(&d_node64, sizeof(double) * 4 * (size_t)n_frames * N_NODES) == cudaSuccess;
  ok = ok && cudaMalloc(&k->d_base, sizeof(double) * (size_t)n_iv * NB * 10) == cudaSuccess;
  ok = ok && cudaMalloc(&k->d_iv_code, sizeof(int) * n_iv) == cudaSuccess;
  ok = ok && cudaMalloc(&k->d_fr_cp, sizeof(float) * n_frames) == cudaSuccess;
  ok = ok && cudaMalloc(&k->d_tmp, sizeof(double) * nd) == cudaSuccess;
  if (!ok) {
    set_error("cudaMalloc failed for kinetics tables");
    cudaFree(d_node64);
    kcs_destroy_kinetics(k);
    return KCS_ERR_OOM;
  }
  std::vector<double> host(nd);
  std::copy(t0.begin(), t0.end(), host.begin());
  std::copy(dt.begin(), dt.end(), host.begin() + n_iv);
  std::copy(gx.begin(), gx.end(), host.begin() + 2 * n_iv);
  std::copy(gw.begin(), gw.end(), host.begin() + 2 * n_iv + NGL);
  std::copy(fdt.begin(), fdt.end(), host.begin() + 2 * n_iv + 2 * NGL);
  KCS_CUDA(cudaMemcpyAsync(k->d_tmp, host.data(), sizeof(double) * nd, cudaMemcpyHostToDevice, s));
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
  ta.base = k->d_base;
  ta.m0 = k->d_tmp + 2 * n_iv + 2 * NGL + n_frames;
  k_tabulate<<<n_iv, NB, 0, s>>>(ta);
  KCS_LAUNCHED();
  k_node_table<<<(N_NODES + 127) / 128, 128, 0, s>>>(k->d_base, ta.iv_dt, k->d_iv_code, n_iv,
                                                       k->d_tmp + 2 * n_iv + 2 * NGL, N_NODES,
                                                       d_node64);
  KCS_LAUNCHED();
  k_cell_table<<<(n_frames * N_CELLS + 127) / 128, 128, 0, s>>>(d_node64, n_frames, N_NODES,
                                                                k->d_cell);
  KCS_LAUNCHED();
  k_frame_tables<<<1, 32, 0, s>>>(ta.m0, k->d_iv_code, n_iv, k->d_tmp + 2 * n_iv + 2 * NGL,
                                  n_frames, k->d_fr_cp);
  KCS_LAUNCHED();
  // the host staging vectors die here: wait for the copies and the tables
  const cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(d_node64);
  if (e != cudaSuccess) {
    set_error("kinetics tables: %s", cudaGetErrorString(e));
    kcs_destroy_kinetics(k);
    return KCS_ERR_CUDA;
  }
  *out = k;
  return KCS_OK;
}

int kcs_destroy_kinetics(kcs_kinetics_t* k) {
  clear_error();
  if (!k) return KCS_OK;
  cudaFree(k->d_cell);
  cudaFree(k->d_base);
  cudaFree(k->d_iv_code);
  cudaFree(k->d_fr_cp);
  cudaFree(k->d_tmp);
  delete k;
  return KCS_OK;
}

int kcs_tac_eval(const kcs_kinetics_t* k, int64_t n_vox, const float* params, float* F, float* J,
                 void* stream) {
  clear_error();
  KCS_REQUIRE(k, "kinetics is NULL");
  KCS_REQUIRE(n_vox >= 0, "n_vox < 0");
  KCS_REQUIRE(n_vox == 0 || (params && F), "NULL argument");
  return launch_tac_eval(k, n_vox, params, F, J, as_stream(stream));
}

int kcs_tac_vjp(const kcs_kinetics_t* k, int64_t n_vox, const float* params, const float* gF,
                float* gparams, void* stream) {
  clear_error();
  KCS_REQUIRE(k, "kinetics is NULL");
  KCS_REQUIRE(n_vox >= 0, "n_vox < 0");
  if (n_vox == 0) return KCS_OK;
  KCS_REQUIRE(params && gF && gparams, "NULL argument");
  const size_t smem = sizeof(float) * TAC_THREADS * (k->M + 1);
  k_tac_vjp<<<(unsigned)((n_vox + TAC_THREADS - 1) / TAC_THREADS), TAC_THREADS, smem,
              as_stream(stream)>>>(k->dev(), n_vox, params, gF, gparams);
  KCS_LAUNCHED();
  return KCS_OK;
}

int kcs_ki(int64_t n_vox, const float* params, float* ki, void* stream) {
  clear_error();
  KCS_REQUIRE(n_vox >= 0, "n_vox < 0");
  if (n_vox == 0) return KCS_OK;
  KCS_REQUIRE(params && ki, "NULL argument");
  k_ki<<<(unsigned)((n_vox + 255) / 256), 256, 0, as_stream(stream)>>>(n_vox, params, ki);
  KCS_LAUNCHED();
  return KCS_OK;
}

int kcs_huber_grad_nb(int nx, int ny, int nz, const float* params, float delta,
                      int neighbourhood, float* grad, void* stream) {
  clear_error();
  KCS_REQUIRE(params && grad, "NULL argument");
  KCS_REQUIRE(nx > 0 && ny > 0 && nz > 0, "sizes must be positive");
  KCS_REQUIRE(delta > 0.f, "delta must be positive");
  KCS_REQUIRE(neighbourhood == 8 || neighbourhood == 26, "neighbourhood %d must be 8 or 26",
              neighbourhood);
  const long long n = (long long)nx * ny * nz;
  k_huber_grad<<<(unsigned)((n + 255) / 256), 256, 0, as_stream(stream)>>>(
      nx, ny, nz, params, delta, neighbourhood == 26 ? 1 : 0, grad);
  KCS_LAUNCHED();
  return KCS_OK;
}

int kcs_huber_grad(int nx, int ny, int nz, const float* params, float delta, float* grad,
                   void* stream) {
  return kcs_huber_grad_nb(nx, ny, nz, params, delta, 8, grad, stream);
}

size_t kcs_lm_workspace_size(int nx, int ny, int nz) {
  if (nx <= 0 || ny <= 0 || nz <= 0) return 0;
  const size_t V = (size_t)nx * ny * nz;
  // ping-pong maps, lambda, two copies of the per-voxel normal equations
  return align256(4 * V * sizeof(float)) + align256(V * sizeof(float)) +
         2 * align256(NE_FIELDS * V * sizeof(float));
}

int kcs_map_lm_fit_ex(const kcs_kinetics_t* k, int nx, int ny, int nz, const void* x,
                      int x_type, const float* x_scale, float* params, float* lambda,
                      int n_steps, float beta_h, float delta, float* F_out, void* workspace,
                      size_t ws_bytes, void* stream) {
  return kcs_map_lm_fit_nb(k, nx, ny, nz, x, x_type, x_scale, params, lambda, n_steps, beta_h,
                           delta, 8, KCS_LM_TAU_DEFAULT, F_out, workspace, ws_bytes, stream);
}

int kcs_map_lm_fit_nb(const kcs_kinetics_t* k, int nx, int ny, int nz, const void* x,
                      int x_type, const float* x_scale, float* params, float* lambda,
                      int n_steps, float beta_h, float delta, int neighbourhood, float tau,
                      float* F_out, void* workspace, size_t ws_bytes, void* stream) {
  clear_error();
  KCS_REQUIRE(tau >= 0.f && tau < 1.f, "tau = %g must lie in [0, 1)", (double)tau);
  KCS_REQUIRE(neighbourhood == 8 || neighbourhood == 26, "neighbourhood %d must be 8 or 26",
              neighbourhood);
  KCS_REQUIRE(k && x && params, "NULL argument");
  KCS_REQUIRE(nx > 0 && ny > 0 && nz > 0, "sizes must be positive");
  KCS_REQUIRE(x_type == KCS_F32 || x_type == KCS_BF16 || x_type == KCS_F16,
              "x_type %d must be KCS_F32, KCS_BF16 or KCS_F16", x_type);
  KCS_REQUIRE(n_steps >= 0, "n_steps < 0");
  KCS_REQUIRE(delta > 0.f && beta_h >= 0.f, "need delta > 0 and beta_h >= 0");
  KCS_REQUIRE(workspace && ws_bytes >= kcs_lm_workspace_size(nx, ny, nz),
              "workspace too small (%zu < %zu)", ws_bytes, kcs_lm_workspace_size(nx, ny, nz));
  cudaStream_t s = as_stream(stream);
  const long long V = (long long)nx * ny * nz;
  char* w = static_cast<char*>(workspace);
  float* pong = reinterpret_cast<float*>(w);
  w += align256(4 * (size_t)V * sizeof(float));
  float* lam_ws = reinterpret_cast<float*>(w);
  w += align256((size_t)V * sizeof(float));
  float* ne_a = reinterpret_cast<float*>(w);
  w += align256(NE_FIELDS * (size_t)V * sizeof(float));
  float* ne_b = reinterpret_cast<float*>(w);
  LmArgs L;
  L.kd = k->dev();
  L.nx = nx; L.ny = ny; L.nz = nz;
  L.x = x;
  L.x_al32 = ((uintptr_t)x & 31u) == 0;
  L.x_scale = x_scale;
  L.lambda = lambda ? lambda : lam_ws;
  L.beta = beta_h;
  L.delta = delta;
  L.tau = tau;
  L.nb3d = neighbourhood == 26 ? 1 : 0;
  L.div_nx = div_magic64((unsigned long long)nx);
  L.div_nxy = div_magic64((unsigned long long)nx * ny);
  const size_t smem = sizeof(float) * LM_BLOCK_VOX * (k->M + 1);
  auto kern = x_type == KCS_BF16 ? k_lm_step<__nv_bfloat16>
            : x_type == KCS_F16 ? k_lm_step<__half> : k_lm_step<float>;
  auto kinit = x_type == KCS_BF16 ? k_lm_normal<__nv_bfloat16>
             : x_type == KCS_F16 ? k_lm_normal<__half> : k_lm_normal<float>;
  for (auto f : {kern, kinit}) {
    KCS_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // Ask for the smallest shared-memory carve-out that holds KCS_LM_MINBLOCKS
    // blocks, leaving the rest of the SM's 256 KB to L1 (coefficient rows).
    KCS_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  KCS_LM_CARVEOUT));
  }
  const unsigned blocks = (unsigned)((V + LM_BLOCK_VOX - 1) / LM_BLOCK_VOX);
  float* cur = params;
  float* nxt = pong;
  float* ne_cur = ne_a;
  float* ne_nxt = ne_b;
  if (n_steps > 0) {
    L.p_in = params;
    L.ne_out = ne_cur;
    kinit<<<blocks, LM_THREADS, smem, s>>>(L);
    KCS_LAUNCHED();
  }
  for (int it = 0; it < n_steps; ++it) {
    L.p_in = cur;
    L.p_out = nxt;
    L.ne_in = ne_cur;
    L.ne_out = ne_nxt;
    L.reset_lambda = (it == 0 && !lambda) ? 1 : 0;
    kern<<<blocks, LM_THREADS, smem, s>>>(L);
    KCS_LAUNCHED();
    std::swap(cur, nxt);
    std::swap(ne_cur, ne_nxt);
  }
  if (cur != params)
    KCS_CUDA(cudaMemcpyAsync(params, cur, 4 * (size_t)V * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (F_out) return launch_tac_eval(k, V, params, F_out, nullptr, s);
  return KCS_OK;
}

int kcs_map_lm_fit(const kcs_kinetics_t* k, int nx, int ny, int nz, const float* x, float* params,
                   float* lambda, int n_steps, float beta_h, float delta, float* F_out,
                   void* workspace, size_t ws_bytes, void* stream) {
  return kcs_map_lm_fit_ex(k, nx, ny, nz, x, KCS_F32, nullptr, params, lambda, n_steps, beta_h,
                           delta, F_out, workspace, ws_bytes, stream);
}

}  // extern "C"

// ---------------------------------------------------------------- no-allocation MAP-LM
// kcs_map_lm_fit_static: the MAP-LM fit with its scratch (ping-pong maps and
// lambda) in a fixed device array owned by this library, for callers that may
// not allocate device memory themselves.  The array lives in every GPU that
// loads the library until the process exits.
namespace {
constexpr size_t kStaticLmBytes =   // the layout of kcs_lm_workspace_size at the maximum size
    ((4 * (size_t)KCS_LM_STATIC_MAX_VOXELS * sizeof(float) + 255) & ~size_t(255)) +
    (((size_t)KCS_LM_STATIC_MAX_VOXELS * sizeof(float) + 255) & ~size_t(255)) +
    2 * (((size_t)NE_FIELDS * KCS_LM_STATIC_MAX_VOXELS * sizeof(float) + 255) & ~size_t(255));
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
  if (stream) {   // the scratch address below belongs to the current device
    int sdev = -1;
    KCS_CUDA(cudaStreamGetDevice(as_stream(stream), &sdev));
    KCS_REQUIRE(sdev == dev, "stream belongs to device %d, the current device is %d", sdev, dev);
  }
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
