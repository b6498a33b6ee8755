// Unfolded OCD with a learnable damping omega_k and regularizer alpha_k per
// sweep (the differentiable form): forward kernel with per-sweep
// checkpoints, hand-written adjoint kernel, and the deterministic reduction
// of the parameter gradients.  See include/ocd.h for the C entry points.
//
// Forward, per (subcarrier w, symbol t) and sweep k = 1..K (Algorithm 1 with
// two changes):
//   d_{u,k} = 1/(||h_u||^2 + alpha_k), p_{u,k} = d_{u,k} ||h_u||^2
//   c = proj(d_{u,k} h_u^H r + p_{u,k} z_u),  dz = omega_k (c - z_u)
//   z_u <- z_u + dz,  r <- r - h_u dz                     (Eq. 15 kept)
// soft output as Eq. 9 with mu~ = p_{u,K}, rho~ = ||h_u||^2 Es / N0[w].
//
// Adjoint of one user update (complex adjoints v' = dl/dRe v + i dl/dIm v;
// primes denote adjoints of the values after the update):
//   g     = z_u' - h_u^H r'                  (adjoint of dz)
//   omega_k'  += Re<c - z_u, g>
//   w'    = mask(omega_k g)                  (mask: 1 strictly inside the box, else 0)
//   z_u'  <- z_u' - omega_k g + p w'
//   r'    <- r' + d h_u w'
//   alpha_k'  += -d^2 Re<h_u^H r, w'> - p d Re<z_u, w'>
// The sweep's inputs (r and z at its start) are checkpointed by the forward
// kernel; the adjoint replays the sweep from its checkpoint (bit-identical
// arithmetic) to recover each update's z_u and h_u^H r, then runs the users
// in reverse.
//
// Layout: one warp per (subcarrier, symbol) sample; lane l holds the
// residual (and its adjoint) of antennas l + 32 j, j < NA; lane u holds z_u,
// ||h_u||^2 and the adjoint of z_u.  When it fits (U (32 NA + 1) complex per
// warp, 4 warps within 192 KB), each warp first copies its sample's channel
// into shared memory, user-major, with coalesced reads, so that every h_u
// load of the K sweeps (and of the adjoint's replays) is a conflict-free
// shared load instead of a strided global one.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <utility>

#include "ocd_common.cuh"
#include "ocd_mma.cuh"
#include "ocd_unfolded.h"

namespace ocd {

namespace {

__device__ __forceinline__ float2 warp_sum2(float2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(kFullMask, v.x, o);
    v.y += __shfl_xor_sync(kFullMask, v.y, o);
  }
  return v;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullMask, v, o);
  return v;
}

__device__ __forceinline__ float2 shfl2(float2 v, int src) {
  return make_float2(__shfl_sync(kFullMask, v.x, src), __shfl_sync(kFullMask, v.y, src));
}

// d and p of sweep k for a user with squared norm n (0, 0 for a zero or
// negative denominator).
__device__ __forceinline__ void gains(float n, float alpha, float& d, float& p) {
  const float den = n + alpha;
  d = den > 0.0f ? 1.0f / den : 0.0f;
  p = d * n;
}

// Binary cross-entropy of a label y in [0, 1] under P(b = 1) = sigmoid(L),
// in the form that cannot overflow: max(L, 0) - y L + log(1 + exp(-|L|)).
__device__ __forceinline__ float bce_term(float L, float y) {
  return fmaxf(L, 0.0f) - y * L + log1pf(expf(-fabsf(L)));
}
// sigmoid(L) = 1 / (1 + exp(-L)), from exp(-|L|) so that it cannot overflow.
__device__ __forceinline__ float sigmoid_of(float L) {
  const float e = expf(-fabsf(L));
  return L >= 0.0f ? 1.0f / (1.0f + e) : e / (1.0f + e);
}

// Soft output of item o = (sample, user): Eq. 9 with mu~ = p and rho~ =
// ||h||^2 Es / n0.  The LLRs go to P.llr when requested and, with the fused
// loss (P.bits), d loss / d L = (sigmoid(L) - y) / N to P.gllr.  Returns the
// item's loss summed over its Q bits in order (0 without the fused loss).
__device__ __forceinline__ float soft_output(const UnfoldParams& P, long long o, float2 z,
                                             float nrm, float p, float n0) {
  DetectParams D = P.D;
  D.rho_scale = P.es / n0;
  const int Q = P.D.Q;
  if (!P.bits) {
    if (P.llr) user_llr(z, nrm, p, D, P.llr + o * Q);
    return 0.0f;
  }
  float* g = P.gllr + o * Q;
  user_llr(z, nrm, p, D, g);  // the LLRs, in the slots of their derivatives
  float acc = 0.0f;
  for (int b = 0; b < Q; ++b) {
    const float L = g[b];
    const float y = __ldg(P.bits + o * Q + b);
    if (P.llr) P.llr[o * Q + b] = L;
    acc += bce_term(L, y);
    g[b] = (sigmoid_of(L) - y) * P.inv_n;
  }
  return acc;
}

// Lane mapping for copying a row-major [n][U] complex array with a warp:
// `rows` = max(1, 32 / U) rows per step, lane -> row r0 (< rows for an
// active lane) and column u.
__device__ __forceinline__ void row_lane(int U, int lane, int& rows, int& r0, int& u) {
  rows = U >= 32 ? 1 : 32 / U;
  r0 = lane / U;
  u = lane - r0 * U;
}

// 8-byte asynchronous copy global -> shared (completed by cp.async.wait_all).
__device__ __forceinline__ void async_copy8(float2* dst, const float2* src) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}

// Column stride (complex elements) of the user-major channel copy in shared
// memory: 32 NA + 1, so the transposing stores of one warp spread over the
// banks and the column loads (lane b reads antenna b) are conflict-free.
template <int NA>
__host__ __device__ constexpr int staged_stride() { return 32 * NA + 1; }

template <int NA, bool SMEM>
struct Warp {
  const UnfoldParams& P;
  const float2* Hw;  // channel of this sample's subcarrier, [B][U] in global memory
  float2* sH;        // SMEM: this warp's user-major copy [U][staged_stride], zero padded
  int lane;

  // Copies H[w] into sH (coalesced reads, transposed stores) and, when ysrc
  // is given, B received values into sy, with asynchronous 8-byte copies
  // (cp.async), so that all of a lane's loads are in flight at once.
  __device__ __forceinline__ void stage(const float2* ysrc = nullptr, float2* sy = nullptr) const {
    if (!SMEM) return;
    constexpr int st = staged_stride<NA>();
    __syncwarp();  // the previous sample's reads are done
    // lane -> (row r0 of a group of `rows` channel rows, user u): the rows
    // of a group are contiguous in H, so each copy instruction reads one
    // contiguous run; no division inside the loop
    int rows, r0, u;
    row_lane(P.U, lane, rows, r0, u);
    if (r0 < rows)
      for (int b = r0; b < P.B; b += rows) async_copy8(sH + u * st + b, Hw + b * P.U + u);
    if (ysrc)
      for (int b = lane; b < P.B; b += 32) async_copy8(sy + b, ysrc + b);
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncwarp();
  }

  __device__ __forceinline__ void load_h(int u, float2 (&h)[NA]) const {
#pragma unroll
    for (int j = 0; j < NA; ++j) {
      const int b = lane + 32 * j;
      if (SMEM) h[j] = sH[u * staged_stride<NA>() + b];  // antennas >= B hold zeros
      else h[j] = b < P.B ? __ldg(Hw + (long long)b * P.U + u) : make_float2(0.0f, 0.0f);
    }
  }

  // lane u (< U) receives ||h_u||^2
  __device__ __forceinline__ float norms() const {
    float mine = 0.0f;
    for (int u = 0; u < P.U; ++u) {
      float2 h[NA];
      load_h(u, h);
      float acc = 0.0f;
#pragma unroll
      for (int j = 0; j < NA; ++j) acc = fmaf(h[j].x, h[j].x, fmaf(h[j].y, h[j].y, acc));
      acc = warp_sum(acc);
      if (lane == u) mine = acc;
    }
    return mine;
  }

  // One forward sweep.  z: lane u holds z_u.  When `keep` is set, lane u
  // records z_u before its update (zb) and h_u^H r at that time (qs).
  template <bool KEEP>
  __device__ __forceinline__ void sweep(float2 (&r)[NA], float2& z, float nrm, float om, float al,
                                        float2& zb, float2& qs) const {
    for (int u = 0; u < P.U; ++u) {
      float2 h[NA];
      load_h(u, h);
      float2 q = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        q.x = fmaf(h[j].x, r[j].x, fmaf(h[j].y, r[j].y, q.x));
        q.y = fmaf(h[j].x, r[j].y, fmaf(-h[j].y, r[j].x, q.y));
      }
      q = warp_sum2(q);
      float d, p;
      gains(__shfl_sync(kFullMask, nrm, u), al, d, p);
      const float2 zu = shfl2(z, u);
      float wr = fmaf(d, q.x, p * zu.x);
      float wi = fmaf(d, q.y, p * zu.y);
      project(wr, wi, P.D);
      const float2 dz = make_float2(om * (wr - zu.x), om * (wi - zu.y));
      if (lane == u) {
        if (KEEP) {
          zb = zu;
          qs = q;
        }
        z = make_float2(zu.x + dz.x, zu.y + dz.y);
      }
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        r[j].x = fmaf(-h[j].x, dz.x, fmaf(h[j].y, dz.y, r[j].x));
        r[j].y = fmaf(-h[j].x, dz.y, fmaf(-h[j].y, dz.x, r[j].y));
      }
    }
  }
};

template <int NA, bool SMEM>
__global__ void __launch_bounds__(128)
ocd_unfolded_forward_kernel(const __grid_constant__ UnfoldParams P) {
  extern __shared__ float2 unf_smem[];
  const int lane = threadIdx.x & 31;
  float2* sH = unf_smem + (threadIdx.x >> 5) * P.U * staged_stride<NA>();
  if (SMEM) {
    // padding antennas (b >= B) stay zero: staging writes only b < B
    for (int i = lane; i < P.U * staged_stride<NA>(); i += 32) sH[i] = make_float2(0.0f, 0.0f);
  }
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  const int stride = P.B + P.U;
  for (long long s = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < P.samples;
       s += nw) {
    const long long w = s / P.T;
    Warp<NA, SMEM> W{P, P.H + w * P.B * P.U, sH, lane};
    W.stage();
    const float nrm = W.norms();
    float2 r[NA];
#pragma unroll
    for (int j = 0; j < NA; ++j) {
      const int b = lane + 32 * j;
      r[j] = b < P.B ? __ldg(P.Y + s * P.B + b) : make_float2(0.0f, 0.0f);
    }
    float2 z = make_float2(0.0f, 0.0f), zb = z, qs = z;
    for (int k = 0; k < P.K; ++k) {
      float2* ck = P.ckpt + ((long long)k * P.samples + s) * stride;
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        const int b = lane + 32 * j;
        if (b < P.B) ck[b] = r[j];
      }
      if (lane < P.U) ck[P.B + lane] = z;
      W.template sweep<false>(r, z, nrm, __ldg(P.omega + k), __ldg(P.alpha + k), zb, qs);
    }
    float lsum = 0.0f;
    if (lane < P.U) {
      const long long o = s * P.U + lane;
      P.xhat[o] = z;
      if (P.llr || P.bits) {
        float d, p;
        gains(nrm, __ldg(P.alpha + P.K - 1), d, p);
        lsum = soft_output(P, o, z, nrm, p, __ldg(P.N0 + w));
      }
    }
    if (P.bits) {
      const float ls = warp_sum(lsum);
      if (lane == 0) P.lpart[s] = ls;
    }
  }
}

// d/dx of sum_b g_b L_b(x) for the bits of one real dimension (Eq. 9 per
// dimension): L_b = rho (min_{bit b = 0} (x - v)^2 - min_{bit b = 1} (x - v)^2)
// is linear in x between changes of the minimizing levels v0*, v1*, with
// slope 2 rho (v1* - v0*).
template <int NB>
__device__ __forceinline__ float dimension_llr_slope_nb(float x, float rho, float step,
                                                        const float* g) {
  constexpr int M = 1 << NB;
  float b0[NB], b1[NB], v0[NB], v1[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) { b0[j] = FLT_MAX; b1[j] = FLT_MAX; v0[j] = 0.0f; v1[j] = 0.0f; }
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const float v = (float)(2 * i + 1 - M) * step;
    const float e = x - v;
    const float dd = e * e;
    const int gw = i ^ (i >> 1);
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      if ((gw >> (NB - 1 - j)) & 1) {
        if (dd < b1[j]) { b1[j] = dd; v1[j] = v; }
      } else {
        if (dd < b0[j]) { b0[j] = dd; v0[j] = v; }
      }
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < NB; ++j) s = fmaf(g[j], 2.0f * rho * (v1[j] - v0[j]), s);
  return s;
}

__device__ __forceinline__ float dimension_llr_slope(float x, float rho, const DetectParams& D,
                                                     const float* g) {
  switch (D.nb) {
    case 1: return dimension_llr_slope_nb<1>(x, rho, D.lvl_step, g);
    case 2: return dimension_llr_slope_nb<2>(x, rho, D.lvl_step, g);
    case 3: return dimension_llr_slope_nb<3>(x, rho, D.lvl_step, g);
    default: return dimension_llr_slope_nb<4>(x, rho, D.lvl_step, g);
  }
}

template <int NA, bool SMEM>
__global__ void __launch_bounds__(128)
ocd_unfolded_backward_kernel(const __grid_constant__ UnfoldParams P) {
  extern __shared__ float2 unf_smem[];
  const int lane = threadIdx.x & 31;
  float2* sH = unf_smem + (threadIdx.x >> 5) * P.U * staged_stride<NA>();
  if (SMEM) {
    // padding antennas (b >= B) stay zero: staging writes only b < B
    for (int i = lane; i < P.U * staged_stride<NA>(); i += 32) sH[i] = make_float2(0.0f, 0.0f);
  }
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  const int stride = P.B + P.U;
  const int K = P.K;
  for (long long s = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < P.samples;
       s += nw) {
    const long long w = s / P.T;
    Warp<NA, SMEM> W{P, P.H + w * P.B * P.U, sH, lane};
    W.stage();
    const float nrm = W.norms();
    // ---- adjoint of the soft output and of xhat (lane u)
    float2 zbar = make_float2(0.0f, 0.0f);
    float al_mu = 0.0f;  // alpha_K' through mu~ = p_{u,K}
    if (lane < P.U) {
      const long long o = s * P.U + lane;
      if (P.dxhat) zbar = __ldg(P.dxhat + o);
      if (P.dllr) {
        float d, p;
        gains(nrm, __ldg(P.alpha + K - 1), d, p);
        if (p > 0.0f) {
          const float2 z = __ldg(P.xhat + o);
          const float rho = nrm * P.es / __ldg(P.N0 + w);
          const float inv = 1.0f / (p * P.D.sqrt_es);
          const float* g = P.dllr + o * P.D.Q;
          const float xr = z.x * inv;
          const float sr = dimension_llr_slope(xr, rho, P.D, g);
          zbar.x += sr * inv;
          float mubar = -sr * xr / p;
          if (!P.D.bpsk) {
            const float xi = z.y * inv;
            const float si = dimension_llr_slope(xi, rho, P.D, g + P.D.nb);
            zbar.y += si * inv;
            mubar -= si * xi / p;
          }
          al_mu = mubar * (-p * d);
        }
      }
    }
    al_mu = warp_sum(al_mu);
    float2 rbar[NA];
#pragma unroll
    for (int j = 0; j < NA; ++j) rbar[j] = make_float2(0.0f, 0.0f);
    float* part = P.partial + s * 2 * K;
    for (int k = K - 1; k >= 0; --k) {
      const float om = __ldg(P.omega + k);
      const float al = __ldg(P.alpha + k);
      // replay sweep k from its checkpoint
      const float2* ck = P.ckpt + ((long long)k * P.samples + s) * stride;
      float2 r[NA];
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        const int b = lane + 32 * j;
        r[j] = b < P.B ? ck[b] : make_float2(0.0f, 0.0f);
      }
      float2 z = lane < P.U ? ck[P.B + lane] : make_float2(0.0f, 0.0f);
      float2 zb = make_float2(0.0f, 0.0f), qs = make_float2(0.0f, 0.0f);
      W.template sweep<true>(r, z, nrm, om, al, zb, qs);
      // reverse over the users
      float om_bar = 0.0f, al_bar = 0.0f;
      for (int u = P.U - 1; u >= 0; --u) {
        float2 h[NA];
        W.load_h(u, h);
        const float2 zu = shfl2(zb, u);
        const float2 q = shfl2(qs, u);
        float d, p;
        gains(__shfl_sync(kFullMask, nrm, u), al, d, p);
        const float wr0 = fmaf(d, q.x, p * zu.x);
        const float wi0 = fmaf(d, q.y, p * zu.y);
        float cr = wr0, ci = wi0;
        project(cr, ci, P.D);
        float mr = 1.0f, mi = 1.0f;
        if (P.D.box) {
          mr = fabsf(wr0) < P.D.box_a ? 1.0f : 0.0f;
          mi = (!P.D.bpsk && fabsf(wi0) < P.D.box_a) ? 1.0f : 0.0f;
        }
        // h_u^H r'
        float2 hr = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int j = 0; j < NA; ++j) {
          hr.x = fmaf(h[j].x, rbar[j].x, fmaf(h[j].y, rbar[j].y, hr.x));
          hr.y = fmaf(h[j].x, rbar[j].y, fmaf(-h[j].y, rbar[j].x, hr.y));
        }
        hr = warp_sum2(hr);
        const float2 zbu = shfl2(zbar, u);
        const float gr = zbu.x - hr.x, gi = zbu.y - hr.y;
        om_bar = fmaf(cr - zu.x, gr, fmaf(ci - zu.y, gi, om_bar));
        const float wbr = mr * om * gr, wbi = mi * om * gi;
        if (lane == u) zbar = make_float2(zbu.x - om * gr + p * wbr, zbu.y - om * gi + p * wbi);
        const float dwr = d * wbr, dwi = d * wbi;
#pragma unroll
        for (int j = 0; j < NA; ++j) {
          rbar[j].x = fmaf(h[j].x, dwr, fmaf(-h[j].y, dwi, rbar[j].x));
          rbar[j].y = fmaf(h[j].x, dwi, fmaf(h[j].y, dwr, rbar[j].y));
        }
        al_bar -= d * d * fmaf(q.x, wbr, q.y * wbi) + p * d * fmaf(zu.x, wbr, zu.y * wbi);
      }
      if (k == K - 1) al_bar += al_mu;
      if (lane == 0) {
        part[2 * k] = om_bar;
        part[2 * k + 1] = al_bar;
      }
    }
  }
}

// out[j] = sum over samples of partial[s][j], j < 2K, in a fixed order,
// times *gscale when it is given.
__global__ void __launch_bounds__(256)
ocd_unfolded_reduce_kernel(const float* __restrict__ partial, long long samples, int K,
                           const float* __restrict__ gscale, float* __restrict__ domega,
                           float* __restrict__ dalpha) {
  __shared__ float red[256];
  pdl_wait();
  const int j = blockIdx.x;  // 0 .. 2K-1
  float acc = 0.0f;
  for (long long s = threadIdx.x; s < samples; s += blockDim.x) acc += partial[s * 2 * K + j];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const float v = gscale ? red[0] * *gscale : red[0];
    if (j & 1) dalpha[j >> 1] = v;
    else domega[j >> 1] = v;
  }
  pdl_trigger();
}

// *loss = scale * (sum over samples of part[s]), in a fixed order.
__global__ void __launch_bounds__(256)
ocd_unfolded_loss_kernel(const float* __restrict__ part, long long samples, float scale,
                         float* __restrict__ loss) {
  __shared__ float red[256];
  pdl_wait();
  float acc = 0.0f;
  for (long long s = threadIdx.x; s < samples; s += blockDim.x) acc += part[s];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = red[0] * scale;
  pdl_trigger();
}

// ---------------------------------------------------------------------------
// Projected arrangement of the same unfolded sweeps (as for detection:
// q = H^H r, q <- q - G[:, u] dz with G = H^H H, identical iterates in exact
// arithmetic).  Lane j (< U) holds q_j, z_j, ||h_j||^2 and their adjoints; a
// user update is one shuffle of dz from lane u and one complex FMA per lane
// with column u of G from shared memory.  The checkpoints are G per sample
// and (q, z) at the start of every sweep.
// ---------------------------------------------------------------------------

// Shared-memory words of one warp: channel copy (U + U%2 rows; the extra row
// stays zero), received vector, G with row stride U + 1.
template <int NA>
__host__ __device__ inline int proj_warp_elems(int U) {
  return (U + (U & 1)) * staged_stride<NA>() + 32 * NA + U * (U + 1);
}

// Checkpoint offsets (complex elements): G of sample s, then (q, z) of
// sweep k for sample s.
__host__ __device__ inline long long ckpt_g(const UnfoldParams& P, long long s) {
  return s * P.U * P.U;
}
__host__ __device__ inline long long ckpt_qz(const UnfoldParams& P, int k, long long s) {
  return P.samples * P.U * P.U + ((long long)k * P.samples + s) * 2 * P.U;
}

// One sweep in q-space.  KEEP: lane u records z_u before its update (zb) and
// q_u at that time (qs).
template <bool KEEP>
__device__ __forceinline__ void qsweep(const UnfoldParams& P, const float2* sG, int gst, int lane,
                                       float2& q, float2& z, float d, float p, float om,
                                       float2& zb, float2& qs) {
  for (int u = 0; u < P.U; ++u) {
    float wr = fmaf(d, q.x, p * z.x);
    float wi = fmaf(d, q.y, p * z.y);
    project(wr, wi, P.D);
    const float2 dz = shfl2(make_float2(om * (wr - z.x), om * (wi - z.y)), u);
    if (lane == u) {
      if (KEEP) {
        zb = z;
        qs = q;
      }
      z = make_float2(z.x + dz.x, z.y + dz.y);
    }
    const float2 g = lane < P.U ? sG[lane * gst + u] : make_float2(0.0f, 0.0f);
    q.x = fmaf(-g.x, dz.x, fmaf(g.y, dz.y, q.x));
    q.y = fmaf(-g.x, dz.y, fmaf(-g.y, dz.x, q.y));
  }
}

// G = H^H H (Hermitian, diagonal real) into sG (row stride U + 1) and
// q0 = H^H y into sy[0 .. U) (over y), from the user-major channel copy sH.
// G: realified m16n8k8 TF32 MMAs with the two-part split (hi*hi, hi*lo +
// lo*hi; FP32-level accuracy).  A k-step covers antennas 4s + t (lane t of a
// quad): A = [Re H^H; Im H^H] of user tile m, B = the same entries of user
// tile n; a diagonal tile skips its lo*hi MMA, the conjugate transpose of
// its hi*lo.  q0 (one received vector: an MMA would use one column of eight)
// by FP32 fmas on the same channel entries: lane (gq, t) sums
// conj(h_{a,u}) y_a over its antennas a = t mod 4 in order, then the four
// lanes of a quad add up as a tree.  UT = user tiles.
// G = H^H H and q0 = H^H y (see gram_q0_tf32) from loaders hld(u, a) (user u,
// antenna a; zero for u >= U is handled here, for a >= B by the loader) and
// yld(a); q0 of user u goes to sq[u].
template <int UT, class HL, class YL>
__device__ __forceinline__ void gram_q0_tf32_impl(HL hld, YL yld, float2* sq, float2* sG, int U,
                                                  int B, int lane) {
  constexpr int NG = UT * (UT + 1) / 2;
  const int gq = lane >> 2, t = lane & 3;
  const int gst = U + 1;
  float g[NG][2][4];
  float2 qf[UT];
#pragma unroll
  for (int i = 0; i < NG; ++i)
#pragma unroll
    for (int e = 0; e < 4; ++e) { g[i][0][e] = 0.0f; g[i][1][e] = 0.0f; }
#pragma unroll
  for (int i = 0; i < UT; ++i) qf[i] = make_float2(0.0f, 0.0f);
  // k-steps in chunks of KC: the loads of a chunk are issued before its
  // products, so that they are in flight together (fewer k-steps per chunk
  // for four user tiles, whose accumulators take most of the registers)
  constexpr int KC = UT >= 4 ? 2 : 8;
  const int nks = (B + 3) / 4;
  for (int ks0 = 0; ks0 < nks; ks0 += KC) {
    const int nc = min(KC, nks - ks0);
    float2 hv[KC][UT], yv[KC];
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      const int a = 4 * (ks0 + c) + t;
#pragma unroll
      for (int m = 0; m < UT; ++m) {
        const int u = m * 8 + gq;
        hv[c][m] = (c < nc && u < U) ? hld(u, a) : make_float2(0.0f, 0.0f);
      }
      yv[c] = c < nc ? yld(a) : make_float2(0.0f, 0.0f);
    }
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      if (c >= nc) break;
      uint32_t ah[UT][3], al[UT][3];
#pragma unroll
      for (int m = 0; m < UT; ++m) {
        split_tf32(hv[c][m].x, ah[m][0], al[m][0]);
        split_tf32(hv[c][m].y, ah[m][2], al[m][2]);
        ah[m][1] = ah[m][2] ^ 0x80000000u;
        al[m][1] = al[m][2] ^ 0x80000000u;
        // q0: conj(h) y
        qf[m].x = fmaf(hv[c][m].x, yv[c].x, fmaf(hv[c][m].y, yv[c].y, qf[m].x));
        qf[m].y = fmaf(hv[c][m].x, yv[c].y, fmaf(-hv[c][m].y, yv[c].x, qf[m].y));
      }
      // round 1: hi*hi and hi*lo of every tile (independent MMAs); round 2:
      // lo*hi, added to a part round 1 updated several MMAs earlier
      int tile = 0;
#pragma unroll
      for (int m = 0; m < UT; ++m) {
#pragma unroll
        for (int n = m; n < UT; ++n, ++tile) {
          mma_tf32(g[tile][0], ah[m][0], ah[m][1], ah[m][2], ah[n][0], ah[n][2]);
          mma_tf32(g[tile][1], ah[m][0], ah[m][1], ah[m][2], al[n][0], al[n][2]);
        }
      }
      // lo*hi off the diagonal only: a diagonal tile's lo*hi is the
      // conjugate transpose of its hi*lo (taken below)
      tile = 0;
#pragma unroll
      for (int m = 0; m < UT; ++m) {
#pragma unroll
        for (int n = m; n < UT; ++n, ++tile)
          if (n != m) mma_tf32(g[tile][1], al[m][0], al[m][1], al[m][2], ah[n][0], ah[n][2]);
      }
    }
  }
  // the quad's partial sums of q0: (t0 + t1) + (t2 + t3)
#pragma unroll
  for (int m = 0; m < UT; ++m) {
    qf[m].x += __shfl_xor_sync(kFullMask, qf[m].x, 1);
    qf[m].y += __shfl_xor_sync(kFullMask, qf[m].y, 1);
    qf[m].x += __shfl_xor_sync(kFullMask, qf[m].x, 2);
    qf[m].y += __shfl_xor_sync(kFullMask, qf[m].y, 2);
  }
  __syncwarp();  // every lane's reads of y are done before q0 can overwrite it
  // diagonal tiles: lo*hi[i][j] = conj(hi*lo[j][i]), read back from sG after
  // the hi*lo parts are written there
  float lhr[UT][2], lhi[UT][2];
  {
    int tile = 0;
#pragma unroll
    for (int m = 0; m < UT; ++m) {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int i = m * 8 + gq, j = m * 8 + 2 * t + e;
        if (i < U && j < U) sG[i * gst + j] = make_float2(g[tile][1][e], g[tile][1][2 + e]);
      }
      tile += UT - m;  // index of the next diagonal tile
    }
    __syncwarp();
#pragma unroll
    for (int m = 0; m < UT; ++m)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int i = m * 8 + gq, j = m * 8 + 2 * t + e;
        const float2 v = (i < U && j < U) ? sG[j * gst + i] : make_float2(0.0f, 0.0f);
        lhr[m][e] = v.x;
        lhi[m][e] = -v.y;
      }
    __syncwarp();
  }
  int tile = 0;
#pragma unroll
  for (int m = 0; m < UT; ++m) {
#pragma unroll
    for (int n = m; n < UT; ++n, ++tile) {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int i = m * 8 + gq, j = n * 8 + 2 * t + e;
        if (i < U && j < U) {
          float re = (n == m ? g[tile][1][e] + lhr[m][e] : g[tile][1][e]) + g[tile][0][e];
          float im = (n == m ? g[tile][1][2 + e] + lhi[m][e] : g[tile][1][2 + e]) + g[tile][0][2 + e];
          if (i == j) im = 0.0f;  // G_uu is real
          sG[i * gst + j] = make_float2(re, im);
          if (n != m) sG[j * gst + i] = make_float2(re, -im);
        }
      }
    }
    const int u = m * 8 + gq;
    if (t == 0 && u < U) sq[u] = qf[m];
  }
}

template <int UT, int NA>
__device__ __forceinline__ void gram_q0_tf32(const float2* sH, float2* sy, float2* sG, int U,
                                             int B, int lane) {
  constexpr int st = staged_stride<NA>();
  gram_q0_tf32_impl<UT>(
      [&](int u, int a) { return sH[u * st + a]; },  // antennas >= B hold zeros
      [&](int a) { return sy[a]; }, sy, sG, U, B, lane);
}

// The same products with H and y read directly from global memory (the
// sample's channel Hw [B][U] and received vector yw [B]); q0 goes to sq.
// A k-step's channel loads cover 4 antenna rows x 8 consecutive users per
// user tile: whole 32-byte sectors.
template <int UT>
__device__ __forceinline__ void gram_q0_tf32_global(const float2* Hw, const float2* yw, float2* sq,
                                                    float2* sG, int U, int B, int lane) {
  gram_q0_tf32_impl<UT>(
      [&](int u, int a) { return a < B ? __ldg(Hw + (long long)a * U + u) : make_float2(0.0f, 0.0f); },
      [&](int a) { return a < B ? __ldg(yw + a) : make_float2(0.0f, 0.0f); }, sq, sG, U, B, lane);
}

// UT: 8-user MMA tiles of the Gram product (1, 2 or 4); one instance each,
// so that a small U does not carry the register budget of 32 users.  Two
// warps per CTA: the per-warp channel copy bounds the warps per SM.
template <int NA, int UT>
__global__ void __launch_bounds__(64)
ocd_unfolded_proj_forward_kernel(const __grid_constant__ UnfoldParams P) {
  extern __shared__ float2 unf_smem[];
  constexpr int st = staged_stride<NA>();
  const int lane = threadIdx.x & 31;
  const int U = P.U, B = P.B;
  const int rows = U + (U & 1);
  const int gst = U + 1;
  float2* sH = unf_smem + (threadIdx.x >> 5) * proj_warp_elems<NA>(U);
  float2* sy = sH + rows * st;
  float2* sG = sy + 32 * NA;
  for (int i = lane; i < rows * st + 32 * NA; i += 32) sH[i] = make_float2(0.0f, 0.0f);
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long s = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < P.samples;
       s += nw) {
    const long long w = s / P.T;
    Warp<NA, true> W{P, P.H + w * B * U, sH, lane};
    W.stage(P.Y + s * B, sy);  // ends with __syncwarp
    // G = H^H H and q0 = H^H y on the tensor cores
    gram_q0_tf32<UT, NA>(sH, sy, sG, U, B, lane);
    __syncwarp();
    float2 q = lane < U ? sy[lane] : make_float2(0.0f, 0.0f);  // q0 (written over y)
    const float nrm = lane < U ? sG[lane * gst + lane].x : 0.0f;
    float2* ckG = P.ckpt + ckpt_g(P, s);
    {
      int rows, r0, u;
      row_lane(U, lane, rows, r0, u);
      if (r0 < rows)
        for (int i = r0; i < U; i += rows) ckG[i * U + u] = sG[i * gst + u];
    }
    float2 z = make_float2(0.0f, 0.0f), zb = z, qs = z;
    for (int k = 0; k < P.K; ++k) {
      if (lane < U) {
        float2* ck = P.ckpt + ckpt_qz(P, k, s);
        ck[lane] = q;
        ck[U + lane] = z;
      }
      float d, p;
      gains(nrm, __ldg(P.alpha + k), d, p);
      qsweep<false>(P, sG, gst, lane, q, z, d, p, __ldg(P.omega + k), zb, qs);
    }
    float lsum = 0.0f;
    if (lane < U) {
      const long long o = s * U + lane;
      P.xhat[o] = z;
      if (P.llr || P.bits) {
        float d, p;
        gains(nrm, __ldg(P.alpha + P.K - 1), d, p);
        lsum = soft_output(P, o, z, nrm, p, __ldg(P.N0 + w));
      }
    }
    if (P.bits) {
      const float ls = warp_sum(lsum);
      if (lane == 0) P.lpart[s] = ls;
    }
    __syncwarp();  // sG and sy are rewritten by the next sample
  }
}

__global__ void __launch_bounds__(128)
ocd_unfolded_proj_backward_kernel(const __grid_constant__ UnfoldParams P) {
  extern __shared__ float2 unf_smem[];
  const int lane = threadIdx.x & 31;
  const int U = P.U;
  const int gst = U + 1;
  const int K = P.K;
  float2* sG = unf_smem + (threadIdx.x >> 5) * U * gst;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long s = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < P.samples;
       s += nw) {
    const long long w = s / P.T;
    __syncwarp();
    const float2* ckG = P.ckpt + ckpt_g(P, s);
    {
      int rows, r0, u;
      row_lane(U, lane, rows, r0, u);
      if (r0 < rows)
        for (int i = r0; i < U; i += rows) sG[i * gst + u] = ckG[i * U + u];
    }
    __syncwarp();
    const float nrm = lane < U ? sG[lane * gst + lane].x : 0.0f;
    // ---- adjoint of the soft output and of xhat (lane u)
    float2 zbar = make_float2(0.0f, 0.0f);
    float al_mu = 0.0f;
    if (lane < U) {
      const long long o = s * U + lane;
      if (P.dxhat) zbar = __ldg(P.dxhat + o);
      if (P.dllr) {
        float d, p;
        gains(nrm, __ldg(P.alpha + K - 1), d, p);
        if (p > 0.0f) {
          const float2 z = __ldg(P.xhat + o);
          const float rho = nrm * P.es / __ldg(P.N0 + w);
          const float inv = 1.0f / (p * P.D.sqrt_es);
          const float* g = P.dllr + o * P.D.Q;
          const float xr = z.x * inv;
          const float sr = dimension_llr_slope(xr, rho, P.D, g);
          zbar.x += sr * inv;
          float mubar = -sr * xr / p;
          if (!P.D.bpsk) {
            const float xi = z.y * inv;
            const float si = dimension_llr_slope(xi, rho, P.D, g + P.D.nb);
            zbar.y += si * inv;
            mubar -= si * xi / p;
          }
          al_mu = mubar * (-p * d);
        }
      }
    }
    al_mu = warp_sum(al_mu);
    float2 qbar = make_float2(0.0f, 0.0f);
    float* part = P.partial + s * 2 * K;
    for (int k = K - 1; k >= 0; --k) {
      const float om = __ldg(P.omega + k);
      float d, p;
      gains(nrm, __ldg(P.alpha + k), d, p);
      float2 q = make_float2(0.0f, 0.0f), z = q;
      if (lane < U) {
        const float2* ck = P.ckpt + ckpt_qz(P, k, s);
        q = ck[lane];
        z = ck[U + lane];
      }
      float2 zb = make_float2(0.0f, 0.0f), qs = zb;
      qsweep<true>(P, sG, gst, lane, q, z, d, p, om, zb, qs);
      float om_l = 0.0f, al_l = 0.0f;  // lane u accumulates the terms of user u
      // hs (lane l) = G[:, l]^H q' = sum_j conj(G[j][l]) q'_j, kept current:
      // an update changes only q'_u (by dq), which adds conj(G[u][l]) dq to
      // every hs_l, so no reduction over the users is needed per update.
      float2 hs = make_float2(0.0f, 0.0f);
      for (int j = 0; j < U; ++j) {
        const float2 qj = shfl2(qbar, j);
        const float2 g = lane < U ? sG[j * gst + lane] : make_float2(0.0f, 0.0f);
        hs.x = fmaf(g.x, qj.x, fmaf(g.y, qj.y, hs.x));
        hs.y = fmaf(g.x, qj.y, fmaf(-g.y, qj.x, hs.y));
      }
      for (int u = U - 1; u >= 0; --u) {
        const float2 hr = hs;  // lane u: G[:, u]^H q'
        float2 dq = make_float2(0.0f, 0.0f);
        if (lane == u) {
          const float wr0 = fmaf(d, qs.x, p * zb.x);
          const float wi0 = fmaf(d, qs.y, p * zb.y);
          float cr = wr0, ci = wi0;
          project(cr, ci, P.D);
          float mr = 1.0f, mi = 1.0f;
          if (P.D.box) {
            mr = fabsf(wr0) < P.D.box_a ? 1.0f : 0.0f;
            mi = (!P.D.bpsk && fabsf(wi0) < P.D.box_a) ? 1.0f : 0.0f;
          }
          const float gr = zbar.x - hr.x, gi = zbar.y - hr.y;
          om_l = fmaf(cr - zb.x, gr, fmaf(ci - zb.y, gi, om_l));
          const float wbr = mr * om * gr, wbi = mi * om * gi;
          zbar = make_float2(zbar.x - om * gr + p * wbr, zbar.y - om * gi + p * wbi);
          dq = make_float2(d * wbr, d * wbi);
          qbar = make_float2(qbar.x + dq.x, qbar.y + dq.y);
          al_l -= d * d * fmaf(qs.x, wbr, qs.y * wbi) + p * d * fmaf(zb.x, wbr, zb.y * wbi);
        }
        dq = shfl2(dq, u);
        const float2 g = lane < U ? sG[u * gst + lane] : make_float2(0.0f, 0.0f);
        hs.x = fmaf(g.x, dq.x, fmaf(g.y, dq.y, hs.x));
        hs.y = fmaf(g.x, dq.y, fmaf(-g.y, dq.x, hs.y));
      }
      float om_bar = warp_sum(om_l);
      float al_bar = warp_sum(al_l);
      if (k == K - 1) al_bar += al_mu;
      if (lane == 0) {
        part[2 * k] = om_bar;
        part[2 * k + 1] = al_bar;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Two samples per warp (U <= 16): lanes 0-15 carry sample 2i, lanes 16-31
// sample 2i + 1, so that every lane of a user update works (one warp per
// sample leaves half of them idle at U = 16).  Lane j = lane % 16 holds q_j,
// z_j, ||h_j||^2 and their adjoints for its half's sample; shuffles stay in
// the half (width 16) and sums run over it.  Per value the operations, and
// the order of every sum, are those of the one-sample kernels above (there
// the upper 16 lanes only ever added zeros), so the results are identical.
// ---------------------------------------------------------------------------

__device__ __forceinline__ float2 shfl2_16(float2 v, int src) {
  return make_float2(__shfl_sync(kFullMask, v.x, src, 16), __shfl_sync(kFullMask, v.y, src, 16));
}
__device__ __forceinline__ float half_sum(float v) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(kFullMask, v, o);
  return v;
}

// qsweep with the lane's half: j = lane % 16, sGh = the half's G.
template <bool KEEP>
__device__ __forceinline__ void qsweep16(const UnfoldParams& P, const float2* sGh, int gst, int j,
                                         float2& q, float2& z, float d, float p, float om,
                                         float2& zb, float2& qs) {
  for (int u = 0; u < P.U; ++u) {
    float wr = fmaf(d, q.x, p * z.x);
    float wi = fmaf(d, q.y, p * z.y);
    project(wr, wi, P.D);
    const float2 dz = shfl2_16(make_float2(om * (wr - z.x), om * (wi - z.y)), u);
    if (j == u) {
      if (KEEP) {
        zb = z;
        qs = q;
      }
      z = make_float2(z.x + dz.x, z.y + dz.y);
    }
    const float2 g = j < P.U ? sGh[j * gst + u] : make_float2(0.0f, 0.0f);
    q.x = fmaf(-g.x, dz.x, fmaf(g.y, dz.y, q.x));
    q.y = fmaf(-g.x, dz.y, fmaf(-g.y, dz.x, q.y));
  }
}

// Shared-memory words of one warp of the paired forward: q0 of the two
// samples (32 each) and their two G.  The channel and the received vector
// are read from global memory by the Gram products (each read once).
__host__ __device__ inline int proj_pair_warp_elems(int U) { return 2 * 32 + 2 * U * (U + 1); }

template <int UT>
__global__ void __launch_bounds__(128)
ocd_unfolded_proj_forward_pair_kernel(const __grid_constant__ UnfoldParams P) {
  extern __shared__ float2 unf_smem[];
  pdl_wait();
  const int lane = threadIdx.x & 31;
  const int U = P.U, B = P.B;
  const int gst = U + 1;
  float2* sq0 = unf_smem + (threadIdx.x >> 5) * proj_pair_warp_elems(U);
  float2* sG0 = sq0 + 2 * 32;
  const int hh = lane >> 4;
  const int j = lane & 15;
  const long long npairs = (P.samples + 1) / 2;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long pi = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); pi < npairs;
       pi += nw) {
    // G = H^H H and q0 = H^H y of both samples, one after the other
    for (int h = 0; h < 2; ++h) {
      const long long s = 2 * pi + h;
      if (s >= P.samples) break;
      float2* sG = sG0 + h * U * gst;
      gram_q0_tf32_global<UT>(P.H + (s / P.T) * B * U, P.Y + s * B, sq0 + 32 * h, sG, U, B, lane);
      __syncwarp();
      float2* ckG = P.ckpt + ckpt_g(P, s);
      int rws, r0, u;
      row_lane(U, lane, rws, r0, u);
      if (r0 < rws)
        for (int i = r0; i < U; i += rws) ckG[i * U + u] = sG[i * gst + u];
    }
    __syncwarp();
    const long long s = 2 * pi + hh;
    const bool valid = s < P.samples;
    const bool act = valid && j < U;
    const float2* sGh = sG0 + hh * U * gst;
    float2 q = act ? sq0[32 * hh + j] : make_float2(0.0f, 0.0f);  // q0
    const float nrm = act ? sGh[j * gst + j].x : 0.0f;
    float2 z = make_float2(0.0f, 0.0f), zb = z, qs = z;
    for (int k = 0; k < P.K; ++k) {
      if (act) {
        float2* ck = P.ckpt + ckpt_qz(P, k, s);
        ck[j] = q;
        ck[U + j] = z;
      }
      float d, p;
      gains(nrm, __ldg(P.alpha + k), d, p);
      qsweep16<false>(P, sGh, gst, j, q, z, d, p, __ldg(P.omega + k), zb, qs);
    }
    float lsum = 0.0f;
    if (act) {
      const long long o = s * U + j;
      P.xhat[o] = z;
      if (P.llr || P.bits) {
        float d, p;
        gains(nrm, __ldg(P.alpha + P.K - 1), d, p);
        lsum = soft_output(P, o, z, nrm, p, __ldg(P.N0 + s / P.T));
      }
    }
    if (P.bits) {
      const float ls = half_sum(lsum);  // over this half's users, in the warp_sum order
      if (j == 0 && valid) P.lpart[s] = ls;
    }
    __syncwarp();  // sG and sq are rewritten by the next pair
  }
  pdl_trigger();
}

__global__ void __launch_bounds__(128)
ocd_unfolded_proj_backward_pair_kernel(const __grid_constant__ UnfoldParams P) {
  extern __shared__ float2 unf_smem[];
  pdl_wait();
  const int lane = threadIdx.x & 31;
  const int U = P.U;
  const int gst = U + 1;
  const int K = P.K;
  const int hh = lane >> 4;
  const int j = lane & 15;
  float2* sG0 = unf_smem + (threadIdx.x >> 5) * 2 * U * gst;
  const long long npairs = (P.samples + 1) / 2;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long pi = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); pi < npairs;
       pi += nw) {
    __syncwarp();
    // both samples' G from the checkpoint: every copy in flight at once
    for (int h = 0; h < 2; ++h) {
      const long long s2 = 2 * pi + h;
      if (s2 >= P.samples) break;
      const float2* ckG = P.ckpt + ckpt_g(P, s2);
      float2* sG = sG0 + h * U * gst;
      int rws, r0, u;
      row_lane(U, lane, rws, r0, u);
      if (r0 < rws)
        for (int i = r0; i < U; i += rws) async_copy8(sG + i * gst + u, ckG + i * U + u);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncwarp();
    const long long s = 2 * pi + hh;
    const bool valid = s < P.samples;
    const bool act = valid && j < U;
    const long long w = valid ? s / P.T : 0;
    const float2* sG = sG0 + hh * U * gst;
    const float nrm = act ? sG[j * gst + j].x : 0.0f;
    // ---- adjoint of the soft output and of xhat (lane j)
    float2 zbar = make_float2(0.0f, 0.0f);
    float al_mu = 0.0f;
    if (act) {
      const long long o = s * U + j;
      if (P.dxhat) zbar = __ldg(P.dxhat + o);
      if (P.dllr) {
        float d, p;
        gains(nrm, __ldg(P.alpha + K - 1), d, p);
        if (p > 0.0f) {
          const float2 z = __ldg(P.xhat + o);
          const float rho = nrm * P.es / __ldg(P.N0 + w);
          const float inv = 1.0f / (p * P.D.sqrt_es);
          const float* g = P.dllr + o * P.D.Q;
          const float xr = z.x * inv;
          const float sr = dimension_llr_slope(xr, rho, P.D, g);
          zbar.x += sr * inv;
          float mubar = -sr * xr / p;
          if (!P.D.bpsk) {
            const float xi = z.y * inv;
            const float si = dimension_llr_slope(xi, rho, P.D, g + P.D.nb);
            zbar.y += si * inv;
            mubar -= si * xi / p;
          }
          al_mu = mubar * (-p * d);
        }
      }
    }
    al_mu = half_sum(al_mu);
    float2 qbar = make_float2(0.0f, 0.0f);
    float* part = P.partial + s * 2 * K;
    // checkpointed (q, z) of the sweep being reversed, loaded one sweep ahead
    float2 nq = make_float2(0.0f, 0.0f), nz = nq;
    if (act) {
      const float2* ck = P.ckpt + ckpt_qz(P, K - 1, s);
      nq = ck[j];
      nz = ck[U + j];
    }
    for (int k = K - 1; k >= 0; --k) {
      const float om = __ldg(P.omega + k);
      float d, p;
      gains(nrm, __ldg(P.alpha + k), d, p);
      float2 q = nq, z = nz;
      if (k > 0 && act) {
        const float2* ck = P.ckpt + ckpt_qz(P, k - 1, s);
        nq = ck[j];
        nz = ck[U + j];
      }
      float2 zb = make_float2(0.0f, 0.0f), qs = zb;
      qsweep16<true>(P, sG, gst, j, q, z, d, p, om, zb, qs);
      float om_l = 0.0f, al_l = 0.0f;  // lane u accumulates the terms of user u
      // hs (lane l) = G[:, l]^H q', kept current as in the one-sample kernel
      float2 hs = make_float2(0.0f, 0.0f);
      for (int i = 0; i < U; ++i) {
        const float2 qi = shfl2_16(qbar, i);
        const float2 g = j < U ? sG[i * gst + j] : make_float2(0.0f, 0.0f);
        hs.x = fmaf(g.x, qi.x, fmaf(g.y, qi.y, hs.x));
        hs.y = fmaf(g.x, qi.y, fmaf(-g.y, qi.x, hs.y));
      }
      // The terms of this lane's user that do not depend on hs, for every
      // lane at once; in the reverse user loop only the chain through hs
      // stays (lane u: g = zbar - G[:, u]^H q', dq = d m om g), and the
      // rest of user u's terms follow the loop.  Per value the operations
      // are those of the one-sample kernel, in the same order.
      const float wr0 = fmaf(d, qs.x, p * zb.x);
      const float wi0 = fmaf(d, qs.y, p * zb.y);
      float cr = wr0, ci = wi0;
      project(cr, ci, P.D);
      float mr = 1.0f, mi = 1.0f;
      if (P.D.box) {
        mr = fabsf(wr0) < P.D.box_a ? 1.0f : 0.0f;
        mi = (!P.D.bpsk && fabsf(wi0) < P.D.box_a) ? 1.0f : 0.0f;
      }
      const float mor = mr * om, moi = mi * om;
      float gr = 0.0f, gi = 0.0f;
      for (int u = U - 1; u >= 0; --u) {
        float2 dq = make_float2(0.0f, 0.0f);
        if (j == u) {
          gr = zbar.x - hs.x;  // hs of lane u: G[:, u]^H q'
          gi = zbar.y - hs.y;
          dq = make_float2(d * (mor * gr), d * (moi * gi));
        }
        dq = shfl2_16(dq, u);
        const float2 g = j < U ? sG[u * gst + j] : make_float2(0.0f, 0.0f);
        hs.x = fmaf(g.x, dq.x, fmaf(g.y, dq.y, hs.x));
        hs.y = fmaf(g.x, dq.y, fmaf(-g.y, dq.x, hs.y));
      }
      if (j < U) {
        om_l = fmaf(cr - zb.x, gr, fmaf(ci - zb.y, gi, om_l));
        const float wbr = mor * gr, wbi = moi * gi;
        zbar = make_float2(zbar.x - om * gr + p * wbr, zbar.y - om * gi + p * wbi);
        const float2 dq = make_float2(d * wbr, d * wbi);
        qbar = make_float2(qbar.x + dq.x, qbar.y + dq.y);
        al_l -= d * d * fmaf(qs.x, wbr, qs.y * wbi) + p * d * fmaf(zb.x, wbr, zb.y * wbi);
      }
      float om_bar = half_sum(om_l);
      float al_bar = half_sum(al_l);
      if (k == K - 1) al_bar += al_mu;
      if (valid && j == 0) {
        part[2 * k] = om_bar;
        part[2 * k + 1] = al_bar;
      }
    }
  }
  pdl_trigger();
}

// cudaFuncSetAttribute once per (device, kernel, size): the launches below
// stay free of attribute calls (and capturable) after the first one.
cudaError_t allow_smem(const void* fn, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  size_t& have = done[{dev, fn}];
  if (have >= smem) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) have = smem;
  return e;
}

// Typed launch with programmatic stream serialization (see pdl_wait): only
// for kernels that call pdl_wait() before their first read of another
// kernel's output.
template <class... Params, class... Args>
cudaError_t launch_pdl(void (*kernel)(Params...), unsigned grid, unsigned block, size_t smem,
                       cudaStream_t stream, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

constexpr int kProjFwdWarps = 2;  // warps per CTA of the projected forward kernel

template <int NA, int UT>
cudaError_t launch_proj_fwd(const UnfoldParams& P, cudaStream_t stream) {
  const size_t smem = (size_t)kProjFwdWarps * proj_warp_elems<NA>(P.U) * sizeof(float2);
  const void* fn = reinterpret_cast<const void*>(ocd_unfolded_proj_forward_kernel<NA, UT>);
  cudaError_t e = allow_smem(fn, smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((P.samples + kProjFwdWarps - 1) / kProjFwdWarps);
  ocd_unfolded_proj_forward_kernel<NA, UT><<<grid, 32 * kProjFwdWarps, smem, stream>>>(P);
  return cudaGetLastError();
}

constexpr int kProjFwdPairWarps = 4;  // warps per CTA of the paired forward kernel

template <int UT>
cudaError_t launch_proj_fwd_pair(const UnfoldParams& P, cudaStream_t stream) {
  const size_t smem = (size_t)kProjFwdPairWarps * proj_pair_warp_elems(P.U) * sizeof(float2);
  const void* fn = reinterpret_cast<const void*>(ocd_unfolded_proj_forward_pair_kernel<UT>);
  cudaError_t e = allow_smem(fn, smem);
  if (e != cudaSuccess) return e;
  const long long npairs = (P.samples + 1) / 2;
  const unsigned grid = (unsigned)((npairs + kProjFwdPairWarps - 1) / kProjFwdPairWarps);
  e = launch_pdl(ocd_unfolded_proj_forward_pair_kernel<UT>, grid, 32 * kProjFwdPairWarps, smem,
                 stream, P);
  return e != cudaSuccess ? e : cudaGetLastError();
}

// U <= 16: two samples per warp; larger U: one sample per warp.
template <int NA>
cudaError_t launch_proj(const UnfoldParams& P, bool backward, unsigned grid, cudaStream_t stream) {
  const bool pair = P.U <= 16;
  if (!backward) {
    if (P.U <= 8) return launch_proj_fwd_pair<1>(P, stream);
    if (P.U <= 16) return launch_proj_fwd_pair<2>(P, stream);
    return launch_proj_fwd<NA, 4>(P, stream);
  }
  const size_t smem = (pair ? 8ull : 4ull) * P.U * (P.U + 1) * sizeof(float2);
  const void* fn = pair ? reinterpret_cast<const void*>(ocd_unfolded_proj_backward_pair_kernel)
                        : reinterpret_cast<const void*>(ocd_unfolded_proj_backward_kernel);
  cudaError_t e = allow_smem(fn, smem);
  if (e != cudaSuccess) return e;
  if (pair) {
    const long long need = ((P.samples + 1) / 2 + 3) / 4;  // 4 warps per CTA, a pair per warp
    if ((long long)grid > need) grid = (unsigned)need;
    e = launch_pdl(ocd_unfolded_proj_backward_pair_kernel, grid, 128, smem, stream, P);
    if (e != cudaSuccess) return e;
  } else {
    ocd_unfolded_proj_backward_kernel<<<grid, 128, smem, stream>>>(P);
  }
  return cudaGetLastError();
}

constexpr size_t kUnfoldedSmemLimit = 192 * 1024;  // per CTA of 4 warps

template <int NA>
cudaError_t launch_pair(const UnfoldParams& P, bool backward, unsigned grid, cudaStream_t stream) {
  const size_t smem = 4ull * P.U * staged_stride<NA>() * sizeof(float2);
  if (smem <= kUnfoldedSmemLimit) {
    const void* fn = backward ? reinterpret_cast<const void*>(ocd_unfolded_backward_kernel<NA, true>)
                              : reinterpret_cast<const void*>(ocd_unfolded_forward_kernel<NA, true>);
    cudaError_t e = allow_smem(fn, smem);
    if (e != cudaSuccess) return e;
    if (backward) ocd_unfolded_backward_kernel<NA, true><<<grid, 128, smem, stream>>>(P);
    else ocd_unfolded_forward_kernel<NA, true><<<grid, 128, smem, stream>>>(P);
  } else {
    if (backward) ocd_unfolded_backward_kernel<NA, false><<<grid, 128, 0, stream>>>(P);
    else ocd_unfolded_forward_kernel<NA, false><<<grid, 128, 0, stream>>>(P);
  }
  return cudaGetLastError();
}

}  // namespace

bool projected_fits(int B, int U) {
  const int na = (B + 31) / 32;
  const int n2 = na <= 1 ? 1 : na <= 2 ? 2 : na <= 4 ? 4 : na <= 8 ? 8 : 16;
  const size_t words = (size_t)(U + (U & 1)) * (32 * n2 + 1) + 32 * n2 + (size_t)U * (U + 1);
  return 4 * words * sizeof(float2) <= kUnfoldedSmemLimit;
}

cudaError_t launch_unfolded(const UnfoldParams& P, bool backward, int sms, cudaStream_t stream) {
  if (P.samples == 0) return cudaSuccess;
  long long grid = (P.samples + 3) / 4;
  const long long cap = (long long)sms * 16;
  if (grid > cap) grid = cap;
  const int na = (P.B + 31) / 32;
  cudaError_t e;
  if (P.projected) {
    if (na <= 1) e = launch_proj<1>(P, backward, (unsigned)grid, stream);
    else if (na <= 2) e = launch_proj<2>(P, backward, (unsigned)grid, stream);
    else if (na <= 4) e = launch_proj<4>(P, backward, (unsigned)grid, stream);
    else if (na <= 8) e = launch_proj<8>(P, backward, (unsigned)grid, stream);
    else e = launch_proj<16>(P, backward, (unsigned)grid, stream);
  } else if (na <= 1) e = launch_pair<1>(P, backward, (unsigned)grid, stream);
  else if (na <= 2) e = launch_pair<2>(P, backward, (unsigned)grid, stream);
  else if (na <= 4) e = launch_pair<4>(P, backward, (unsigned)grid, stream);
  else if (na <= 8) e = launch_pair<8>(P, backward, (unsigned)grid, stream);
  else e = launch_pair<16>(P, backward, (unsigned)grid, stream);
  if (e != cudaSuccess) return e;
  if (!backward) {
    if (!P.bits) return e;
    e = launch_pdl(ocd_unfolded_loss_kernel, 1, 256, 0, stream, (const float*)P.lpart,
                   P.samples, P.inv_n, P.loss);
    return e != cudaSuccess ? e : cudaGetLastError();
  }
  e = launch_pdl(ocd_unfolded_reduce_kernel, (unsigned)(2 * P.K), 256, 0, stream,
                 (const float*)P.partial, P.samples, P.K, P.gscale, P.domega, P.dalpha);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace ocd

// ---------------------------------------------------------------------------
// C entry points
// ---------------------------------------------------------------------------
#include <math.h>
#include <string.h>

#include "ocd.h"
#include "ocd_host.h"

using namespace ocdh;

namespace {

// OCD_ALGO_AUTO takes the projected arrangement whenever its shared-memory
// copy fits (every shape up to 512 x 32 except the largest B with large U).
int resolve_unfolded_algo(int algo, int B, int U) {
  if (algo == OCD_ALGO_AUTO) return ocd::projected_fits(B, U) ? OCD_ALGO_PROJECTED : OCD_ALGO_RESIDUAL;
  return algo;
}

int unfolded_common(const void* H, int Nsc, int B, int U, int T, const float* N0, float Es,
                    int K, int mode, int qam_order, const float* omega, const float* alpha,
                    const void* xhat, const void* ckpt, int algo, ocd::UnfoldParams& P) {
  Alphabet al;
  if (algo != OCD_ALGO_AUTO && algo != OCD_ALGO_RESIDUAL && algo != OCD_ALGO_PROJECTED)
    return fail(OCD_ERR_ARG, "unknown algo %d", algo);
  if (Nsc < 0 || T < 0) return fail(OCD_ERR_ARG, "Nsc=%d and T=%d must be >= 0", Nsc, T);
  if (B < 1 || B > OCD_MAX_ANTENNAS) return fail(OCD_ERR_ARG, "B=%d outside 1..%d", B, OCD_MAX_ANTENNAS);
  if (U < 1 || U > OCD_MAX_USERS) return fail(OCD_ERR_ARG, "U=%d outside 1..%d", U, OCD_MAX_USERS);
  if (K < 1 || K > OCD_MAX_SWEEPS) return fail(OCD_ERR_ARG, "K=%d outside 1..%d", K, OCD_MAX_SWEEPS);
  if (mode != OCD_MMSE && mode != OCD_BOX) return fail(OCD_ERR_ARG, "unknown mode %d", mode);
  if (!alphabet_of(qam_order, al)) return fail(OCD_ERR_ARG, "unsupported qam_order %d", qam_order);
  if (!(Es > 0.0f) || !isfinite(Es)) return fail(OCD_ERR_ARG, "Es must be finite and > 0");
  const long long samples = (long long)Nsc * T;
  if (samples > 0 && (!H || !N0 || !omega || !alpha || !xhat || !ckpt))
    return fail(OCD_ERR_ARG, "H, N0, omega, alpha, xhat and ckpt must not be NULL");
  if ((((uintptr_t)H | (uintptr_t)xhat | (uintptr_t)ckpt) & 7u) ||
      (((uintptr_t)N0 | (uintptr_t)omega | (uintptr_t)alpha) & 3u))
    return fail(OCD_ERR_ARG, "arrays must be aligned to their element size");
  memset(&P, 0, sizeof(P));
  build_params(H, nullptr, OCD_STORE_C64, Nsc, B, U, T, 1.0f, Es, K, mode, al, const_cast<void*>(xhat),
               nullptr, P.D);
  P.H = static_cast<const float2*>(H);
  P.N0 = N0;
  P.omega = omega;
  P.alpha = alpha;
  P.xhat = static_cast<float2*>(const_cast<void*>(xhat));
  P.ckpt = static_cast<float2*>(const_cast<void*>(ckpt));
  P.samples = samples;
  P.Nsc = Nsc; P.B = B; P.U = U; P.T = T; P.K = K;
  P.es = Es;
  algo = resolve_unfolded_algo(algo, B, U);
  if (algo == OCD_ALGO_PROJECTED && !ocd::projected_fits(B, U))
    return fail(OCD_ERR_UNSUPPORTED, "projected unfolded form: B=%d U=%d exceeds shared memory", B, U);
  P.projected = algo == OCD_ALGO_PROJECTED;
  return OCD_OK;
}

int sms_of_current(int& sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  DeviceInfo di;
  const int st = device_info(dev, di);
  if (st != OCD_OK) return st;
  sms = di.sms;
  return OCD_OK;
}

// Adjoint and reduction; gscale (device float or null) multiplies the summed
// parameter gradients.
int unfolded_backward(const void* H, int Nsc, int B, int U, int T, const float* N0, float Es,
                      int K, int mode, int qam_order, const float* omega, const float* alpha,
                      const void* xhat, const void* ckpt, const void* dxhat, const float* dllr,
                      const float* gscale, float* domega, float* dalpha, void* workspace,
                      size_t workspace_bytes, int algo, cudaStream_t stream);

}  // namespace

extern "C" {

size_t ocd_unfolded_checkpoint_size(int Nsc, int B, int U, int T, int K, int algo) {
  if (Nsc <= 0 || T <= 0 || B <= 0 || U <= 0 || K <= 0) return 0;
  const size_t S = (size_t)Nsc * T;
  if (resolve_unfolded_algo(algo, B, U) == OCD_ALGO_PROJECTED)
    return (S * U * U + (size_t)K * S * 2 * U) * sizeof(float2);
  return (size_t)K * S * (B + U) * sizeof(float2);
}

size_t ocd_unfolded_workspace_size(int Nsc, int T, int K) {
  if (Nsc <= 0 || T <= 0 || K <= 0) return 0;
  const size_t b = (size_t)Nsc * T * 2 * K * sizeof(float);
  return (b + 255) / 256 * 256;
}

int ocd_unfolded_forward(const void* H, const void* Y, int Nsc, int B, int U, int T,
                         const float* N0, float Es, int K, int mode, int qam_order,
                         const float* omega, const float* alpha, void* xhat, float* llr,
                         void* ckpt, int algo, cudaStream_t stream) {
  ocd::UnfoldParams P;
  int st = unfolded_common(H, Nsc, B, U, T, N0, Es, K, mode, qam_order, omega, alpha, xhat, ckpt,
                           algo, P);
  if (st != OCD_OK) return st;
  if (P.samples > 0 && !Y) return fail(OCD_ERR_ARG, "Y must not be NULL");
  if (((uintptr_t)Y & 7u) || ((uintptr_t)llr & 3u))
    return fail(OCD_ERR_ARG, "arrays must be aligned to their element size");
  if (P.samples == 0) return OCD_OK;
  P.Y = static_cast<const float2*>(Y);
  P.llr = llr;
  int sms = 0;
  st = sms_of_current(sms);
  if (st != OCD_OK) return st;
  const cudaError_t e = ocd::launch_unfolded(P, false, sms, stream);
  if (e != cudaSuccess) return cuda_fail(e, "unfolded forward launch");
  return OCD_OK;
}

int ocd_unfolded_backward(const void* H, int Nsc, int B, int U, int T, const float* N0,
                          float Es, int K, int mode, int qam_order, const float* omega,
                          const float* alpha, const void* xhat, const void* ckpt,
                          const void* dxhat, const float* dllr, float* domega, float* dalpha,
                          void* workspace, size_t workspace_bytes, int algo, cudaStream_t stream) {
  return unfolded_backward(H, Nsc, B, U, T, N0, Es, K, mode, qam_order, omega, alpha, xhat, ckpt,
                           dxhat, dllr, nullptr, domega, dalpha, workspace, workspace_bytes, algo,
                           stream);
}

int ocd_unfolded_bce_forward(const void* H, const void* Y, int Nsc, int B, int U, int T,
                             const float* N0, float Es, int K, int mode, int qam_order,
                             const float* omega, const float* alpha, const float* bits,
                             void* xhat, float* llr, float* dllr, float* loss, void* ckpt,
                             void* workspace, size_t workspace_bytes, int algo,
                             cudaStream_t stream) {
  ocd::UnfoldParams P;
  int st = unfolded_common(H, Nsc, B, U, T, N0, Es, K, mode, qam_order, omega, alpha, xhat, ckpt,
                           algo, P);
  if (st != OCD_OK) return st;
  if (!loss) return fail(OCD_ERR_ARG, "loss must not be NULL");
  if (P.samples > 0 && (!Y || !bits || !dllr))
    return fail(OCD_ERR_ARG, "Y, bits and dllr must not be NULL");
  if (((uintptr_t)Y & 7u) || (((uintptr_t)llr | (uintptr_t)bits | (uintptr_t)dllr |
                               (uintptr_t)loss | (uintptr_t)workspace) & 3u))
    return fail(OCD_ERR_ARG, "arrays must be aligned to their element size");
  if (P.samples == 0) {
    const cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    return OCD_OK;
  }
  if (!workspace || workspace_bytes < ocd_unfolded_workspace_size(Nsc, T, K))
    return fail(OCD_ERR_ARG, "workspace of %zu bytes is smaller than the %zu needed",
                workspace_bytes, ocd_unfolded_workspace_size(Nsc, T, K));
  P.Y = static_cast<const float2*>(Y);
  P.llr = llr;
  P.bits = bits;
  P.gllr = dllr;
  P.lpart = static_cast<float*>(workspace);
  P.loss = loss;
  P.inv_n = (float)(1.0 / ((double)P.samples * U * P.D.Q));
  int sms = 0;
  st = sms_of_current(sms);
  if (st != OCD_OK) return st;
  const cudaError_t e = ocd::launch_unfolded(P, false, sms, stream);
  if (e != cudaSuccess) return cuda_fail(e, "unfolded forward launch");
  return OCD_OK;
}

int ocd_unfolded_bce_backward(const void* H, int Nsc, int B, int U, int T, const float* N0,
                              float Es, int K, int mode, int qam_order, const float* omega,
                              const float* alpha, const void* xhat, const void* ckpt,
                              const float* dllr, const float* dloss, float* domega,
                              float* dalpha, void* workspace, size_t workspace_bytes, int algo,
                              cudaStream_t stream) {
  if ((long long)Nsc * T > 0 && !dllr) return fail(OCD_ERR_ARG, "dllr must not be NULL");
  if ((uintptr_t)dloss & 3u) return fail(OCD_ERR_ARG, "arrays must be aligned to their element size");
  return unfolded_backward(H, Nsc, B, U, T, N0, Es, K, mode, qam_order, omega, alpha, xhat, ckpt,
                           nullptr, dllr, dloss, domega, dalpha, workspace, workspace_bytes, algo,
                           stream);
}

}  // extern "C"

namespace {

int unfolded_backward(const void* H, int Nsc, int B, int U, int T, const float* N0, float Es,
                      int K, int mode, int qam_order, const float* omega, const float* alpha,
                      const void* xhat, const void* ckpt, const void* dxhat, const float* dllr,
                      const float* gscale, float* domega, float* dalpha, void* workspace,
                      size_t workspace_bytes, int algo, cudaStream_t stream) {
  ocd::UnfoldParams P;
  int st = unfolded_common(H, Nsc, B, U, T, N0, Es, K, mode, qam_order, omega, alpha, xhat, ckpt,
                           algo, P);
  if (st != OCD_OK) return st;
  if (!domega || !dalpha) return fail(OCD_ERR_ARG, "domega and dalpha must not be NULL");
  if (((uintptr_t)dxhat & 7u) || (((uintptr_t)dllr | (uintptr_t)domega | (uintptr_t)dalpha |
                                   (uintptr_t)workspace) & 3u))
    return fail(OCD_ERR_ARG, "arrays must be aligned to their element size");
  if (P.samples > 0 && (!workspace || workspace_bytes < ocd_unfolded_workspace_size(Nsc, T, K)))
    return fail(OCD_ERR_ARG, "workspace of %zu bytes is smaller than the %zu needed",
                workspace_bytes, ocd_unfolded_workspace_size(Nsc, T, K));
  cudaError_t e;
  if (P.samples == 0) {
    e = cudaMemsetAsync(domega, 0, K * sizeof(float), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(dalpha, 0, K * sizeof(float), stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    return OCD_OK;
  }
  P.dxhat = static_cast<const float2*>(dxhat);
  P.dllr = dllr;
  P.gscale = gscale;
  P.partial = static_cast<float*>(workspace);
  P.domega = domega;
  P.dalpha = dalpha;
  int sms = 0;
  st = sms_of_current(sms);
  if (st != OCD_OK) return st;
  e = ocd::launch_unfolded(P, true, sms, stream);
  if (e != cudaSuccess) return cuda_fail(e, "unfolded backward launch");
  return OCD_OK;
}

}  // namespace
