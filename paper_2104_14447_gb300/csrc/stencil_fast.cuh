// stencil_fast.cuh -- warp-per-target GMLS stencils, FP32 QR + float-float refinement.
// (kernel template; the instantiations live in fast_*.cu, the dispatch in
// stencil_fast.cu)
//
// Same mathematics as stencil.cu (Sec. 2.1 / 2.2 / 2.5 of the paper: weighted,
// eps-scaled basis matrix B = sqrt(W) P, least-squares solve through a
// Householder QR, functional rows lambda, weights w = sqrt(W) Q R^{-T}
// lambda^T), laid out for GB300:
//
//  * one warp owns one target; lane l holds rows l, l+32, ... of the FP32
//    QR tile in registers (compile-time basis size N and rows-per-lane MR, so
//    the factorisation is fully unrolled); padded rows are zero and exactly
//    neutral for Householder reflections;
//  * the tile B is built directly in float-float (hi + lo, ~48 bits) from
//    float-float coordinates, so no FP64 instruction runs in the hot loop;
//  * refinement of the augmented system [[I, B], [B^T, 0]] [s; -y] =
//    [0; lambda^T] (Bjorck) computes its residuals f = B y - s and
//    g = lambda - B^T s with compensated float-float dot products and its
//    corrections with the FP32 factors;
//  * w = sqrt(W) s is rounded to FP64 only when stored.
//
// Targets this path does not cover (Neumann constraint, a basis size other
// than the instantiation's, more rows than the tile holds, an ill-conditioned
// FP32 factor or a refinement that misses its tolerance) are appended to the
// redo list for the FP64 kernel.
#pragma once
#include <cuda_runtime.h>

#include <utility>

#include "basis_tables.cuh"
#include "ff.cuh"
#include "gmls_internal.cuh"

namespace gmls {

template <int MR, int N>
struct FastLay {
  static constexpr int LD = 32 * MR + 1;  // odd: column walks by different lanes avoid bank conflicts
  static constexpr int RS = N | 1;        // odd row stride of the staged triangular factor
  static constexpr size_t B = 0;                                // ff [N][LD]
  static constexpr size_t SW = B + sizeof(ff) * N * LD;         // ff [LD]  sqrt(W) per row
  static constexpr size_t R = SW + sizeof(ff) * LD;             // float [N][RS] R (upper)
  static constexpr size_t ID = R + sizeof(float) * N * RS;      // float [N] 1 / r_ii
  static constexpr size_t TAU = ID + sizeof(float) * N;         // float [N]
  static constexpr size_t PART = TAU + sizeof(float) * N;       // ff [32] partial sums
  static constexpr size_t S = PART + sizeof(ff) * 32;           // ff [L][LD] s iterates
  // the rest depends on the number of solve rows L
  __host__ __device__ static size_t Y(int L) { return S + sizeof(ff) * L * LD; }      // ff [L][N]
  __host__ __device__ static size_t LAM(int L) { return Y(L) + sizeof(ff) * L * N; }  // ff [L][N]
  __host__ __device__ static size_t G(int L) { return LAM(L) + sizeof(ff) * L * N; }  // float [L][N]
  __host__ __device__ static size_t bytes(int L) { return (G(L) + sizeof(float) * L * N + 15) & ~size_t(15); }
};

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float wmax(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// apply Q (REV: H_0 ... H_{N-1} z, i.e. reflectors in reverse order) or Q^T
// to the row-distributed vectors z[l][i], l < L
// All-reduce over the warp of v[B..N) (compile-time range): recursive halving
// (each lane keeps the half of the values picked by its lane bit and adds its
// partner's copy of that half) until every lane holds one total, butterflies
// over the remaining lanes, then a broadcast of each total.  About 2(N - B)
// shuffles instead of 5(N - B) for independent butterflies.
template <int N, int B>
__device__ __forceinline__ void allreduce_tail(float (&v)[N], int lane) {
  constexpr int C = N - B;
  if constexpr (C <= 0) {
    return;
  } else if constexpr (C <= 2) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int c = B; c < N; ++c) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
  } else {
    constexpr int P = C <= 4 ? 4 : C <= 8 ? 8 : C <= 16 ? 16 : 32;
    float w[P];
#pragma unroll
    for (int i = 0; i < P; ++i) w[i] = (i < C) ? v[B + (i < C ? i : 0)] : 0.0f;
    // halving: stage with offset o keeps P/2^s values; the kept half is the
    // upper one on lanes whose bit o is set
    int m = P;
#pragma unroll
    for (int o = 16; o > 0 && m > 1; o >>= 1) {
      const bool up = (lane & o) != 0;
      const int h = m >> 1;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        if (i < h) {
          const float send = up ? w[i] : w[i + h];
          const float keep = up ? w[i + h] : w[i];
          w[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
      }
      m = h;
    }
    // lanes sharing a value index add up across the remaining lane bits
    constexpr int used = P == 4 ? 2 : P == 8 ? 3 : P == 16 ? 4 : 5;  // stages done
#pragma unroll
    for (int o = 16 >> used; o > 0; o >>= 1) w[0] += __shfl_xor_sync(0xffffffffu, w[0], o);
    // value index held by a lane: its top `used` bits (offsets 16, 8, ...)
#pragma unroll
    for (int i = 0; i < C; ++i) {
      // the lane whose top bits spell i (others bits zero) holds total i
      const int src = i << (5 - used);
      v[B + i] = __shfl_sync(0xffffffffu, w[0], src);
    }
  }
}

// One Householder step on column KC of the register tile: reflector from
// rows > KC, then the trailing columns (dot products all-reduced together).
template <int MR, int N, int KC>
__device__ __forceinline__ void qr_column(float (&a)[MR][N], float* tau, int lane) {
  float sig = 0.0f;
#pragma unroll
  for (int i = 0; i < MR; ++i)
    if (lane + 32 * i > KC) sig = fmaf(a[i][KC], a[i][KC], sig);
  sig = wsum(sig);
  const float alpha = __shfl_sync(0xffffffffu, a[KC / 32][KC], KC % 32);
  float tk = 0.0f, beta = alpha;
  if (sig > 0.0f) {
    const float nrm = sqrtf(fmaf(alpha, alpha, sig));
    beta = alpha >= 0.0f ? -nrm : nrm;
    const float scale = 1.0f / (alpha - beta);
    tk = (beta - alpha) / beta;
#pragma unroll
    for (int i = 0; i < MR; ++i)
      if (lane + 32 * i > KC) a[i][KC] *= scale;
  }
  if (lane == KC % 32) a[KC / 32][KC] = beta;
  if (lane == 0) tau[KC] = tk;
  float v[MR];
#pragma unroll
  for (int i = 0; i < MR; ++i) {
    const int r = lane + 32 * i;
    v[i] = (r > KC) ? a[i][KC] : (r == KC ? 1.0f : 0.0f);
  }
  float dots[N];
#pragma unroll
  for (int c = KC + 1; c < N; ++c) {
    float p = 0.0f;
#pragma unroll
    for (int i = 0; i < MR; ++i) p = fmaf(v[i], a[i][c], p);
    dots[c] = p;
  }
  allreduce_tail<N, KC + 1>(dots, lane);
#pragma unroll
  for (int c = KC + 1; c < N; ++c) {
    const float tc = dots[c] * tk;
#pragma unroll
    for (int i = 0; i < MR; ++i) a[i][c] = fmaf(-tc, v[i], a[i][c]);
  }
}

template <int MR, int N, int... K>
__device__ __forceinline__ void qr_columns(float (&a)[MR][N], float* tau, int lane, std::integer_sequence<int, K...>) {
  (qr_column<MR, N, K>(a, tau, lane), ...);
}

template <int MR, int N, int L, bool REV>
__device__ __forceinline__ void apply_q_regs(const float (&a)[MR][N], const float* tau, float (&z)[L][MR], int lane) {
#pragma unroll
  for (int s = 0; s < N; ++s) {
    const int k = REV ? N - 1 - s : s;
    const float tk = tau[k];
    float v[MR];
#pragma unroll
    for (int i = 0; i < MR; ++i) {
      const int r = lane + 32 * i;
      v[i] = (r > k) ? a[i][k] : (r == k ? 1.0f : 0.0f);
    }
    float d[L];
#pragma unroll
    for (int l = 0; l < L; ++l) {
      d[l] = 0.0f;
#pragma unroll
      for (int i = 0; i < MR; ++i) d[l] = fmaf(v[i], z[l][i], d[l]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int l = 0; l < L; ++l) d[l] += __shfl_xor_sync(0xffffffffu, d[l], o);
#pragma unroll
    for (int l = 0; l < L; ++l) {
      const float dl = d[l] * tk;
#pragma unroll
      for (int i = 0; i < MR; ++i) z[l][i] = fmaf(-dl, v[i], z[l][i]);
    }
  }
}

// w <- R^{-T} w (forward substitution), w[l][t] holds entry p = lane + 32 t
template <int N, int L>
__device__ __forceinline__ void solve_rt_lanes(const float* Rs, int RS, const float* idg, float (&w)[L][(N + 31) / 32],
                                               int lane) {
  constexpr int NT = (N + 31) / 32;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const float inv = idg[i];
#pragma unroll
    for (int l = 0; l < L; ++l) {
      const float yi = __shfl_sync(0xffffffffu, w[l][i / 32], i % 32) * inv;
      if (lane == i % 32) w[l][i / 32] = yi;
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const int p = lane + 32 * t;
        if (p > i && p < N) w[l][t] = fmaf(-Rs[i * RS + p], yi, w[l][t]);
      }
    }
  }
}

// w <- R^{-1} w (back substitution)
template <int N, int L>
__device__ __forceinline__ void solve_r_lanes(const float* Rs, int RS, const float* idg, float (&w)[L][(N + 31) / 32],
                                              int lane) {
  constexpr int NT = (N + 31) / 32;
#pragma unroll
  for (int i = N - 1; i >= 0; --i) {
    const float inv = idg[i];
#pragma unroll
    for (int l = 0; l < L; ++l) {
      const float yi = __shfl_sync(0xffffffffu, w[l][i / 32], i % 32) * inv;
      if (lane == i % 32) w[l][i / 32] = yi;
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const int p = lane + 32 * t;
        if (p < i) w[l][t] = fmaf(-Rs[p * RS + i], yi, w[l][t]);
      }
    }
  }
}

template <int KIND, int D, int DEG, int MR, int L>
__global__ void __launch_bounds__(128) stencil_fast_kernel(StencilJob j) {
  constexpr int N = gmls_gen::basis_size(KIND, D, DEG);
  constexpr int NC = (KIND == GMLS_BASIS_SCALAR) ? 1 : D;
  constexpr int ROWS = 32 * MR;
  constexpr int NT = (N + 31) / 32;
  using Lay = FastLay<MR, N>;
  constexpr int LD = Lay::LD, RS = Lay::RS;
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  unsigned char* base = smem + (size_t)warp * Lay::bytes(L);
  ff* Bs = reinterpret_cast<ff*>(base + Lay::B);
  ff* SWs = reinterpret_cast<ff*>(base + Lay::SW);
  ff* Ss = reinterpret_cast<ff*>(base + Lay::S);
  ff* Ys = reinterpret_cast<ff*>(base + Lay::Y(L));
  ff* LAMs = reinterpret_cast<ff*>(base + Lay::LAM(L));
  float* Rs = reinterpret_cast<float*>(base + Lay::R);
  float* IDs = reinterpret_cast<float*>(base + Lay::ID);
  float* TAUs = reinterpret_cast<float*>(base + Lay::TAU);
  float* Gs = reinterpret_cast<float*>(base + Lay::G(L));
  ff* PARTs = reinterpret_cast<ff*>(base + Lay::PART);
  const int64_t n = j.n;
  const int64_t n_items = j.items ? (int64_t)(*j.n_items) : j.n_tgt;
  const float tolf = (float)j.tol;

  for (int64_t it = (int64_t)blockIdx.x * wpb + warp; it < n_items; it += (int64_t)gridDim.x * wpb) {
    const int64_t to = j.items ? (int64_t)j.items[it] : it;
    const int64_t t = j.tgt[to];
    const int64_t o0 = j.off[to];
    const int k = (int)(j.off[to + 1] - o0);
    const int M = k * NC;
    uint8_t st = j.nbr_status ? j.nbr_status[to] : 0;
    const bool neu = j.neumann && j.bflag && j.bflag[t];
    const bool too_few = (st & GMLS_T_TOO_FEW_NEIGHBOURS) || k <= 0 || !(j.eps[to] > 0.0);
    if (!too_few && (neu || M > ROWS || M < N)) {
      // not for this path: the FP64 kernel takes it (and writes every output)
      if (lane == 0) {
        const int slot = atomicAdd(j.fb_count, 1);
        j.fb_items[slot] = (int32_t)to;
        j.status[to] = 0;
      }
      continue;
    }
    if (too_few) {
      for (int f = 0; f < j.nout; ++f) {
        const int64_t cnt = (int64_t)j.out_rows[f] * k * j.out_ncomp[f];
        double* w = j.out_w[f] + o0 * (int64_t)j.out_rows[f] * j.out_ncomp[f];
        for (int64_t e = lane; e < cnt; e += 32) w[e] = 0.0;
      }
      if (j.beta)
        for (int l = lane; l < L; l += 32) j.beta[to * L + l] = 0.0;
      if (lane == 0) {
        j.status[to] = st;
        if (j.iters) j.iters[to] = 0;
      }
      continue;
    }

    // ---- 1. float-float tile B = sqrt(W) P, rows (neighbour, component)
    const ff eps(j.eps[to]);
    const ff inv_eps = recip(eps);
    float xth[3] = {0.f, 0.f, 0.f}, xtl[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int c = 0; c < D; ++c) {
      xth[c] = j.xh[c * n + t];
      xtl[c] = j.xl[c * n + t];
    }
    const int half_p = j.wpow_half;
    for (int q = lane; q < ROWS / NC; q += 32) {
      if (q < k) {
        const int32_t jj = j.idx[o0 + q];
        ff dx[3], xi[3];
        ff r2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < D; ++c) {
          dx[c] = sub_pair(j.xh[c * n + jj], j.xl[c * n + jj], xth[c], xtl[c]);
          xi[c] = dx[c] * inv_eps;
          r2 = r2 + dx[c] * dx[c];
        }
        const ff u = ff(1.f, 0.f) - sqrt_ff(r2) * inv_eps;
        ff sw(0.f, 0.f);
        if (u.h > 0.0f) {
          sw = u;
          for (int p = 1; p < half_p; ++p) sw = sw * u;
        }
        gmls_gen::BasisEval<KIND, D, DEG>::template run<ff>(xi, Bs + q * NC, LD, sw);
#pragma unroll
        for (int c = 0; c < NC; ++c) SWs[q * NC + c] = sw;
      } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          SWs[q * NC + c] = ff(0.f, 0.f);
#pragma unroll
          for (int i = 0; i < N; ++i) Bs[i * LD + q * NC + c] = ff(0.f, 0.f);
        }
      }
    }
    // rows past the last whole neighbour (ROWS not a multiple of NC)
    for (int r = (ROWS / NC) * NC + lane; r < ROWS; r += 32) {
      SWs[r] = ff(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < N; ++i) Bs[i * LD + r] = ff(0.f, 0.f);
    }
    // functional rows (float-float), lanes over (row, column)
    for (int e = lane; e < L * N; e += 32) {
      const int l = e / N, i = e % N;
      ff f(gmls_gen::lam_coef_f(KIND, D, DEG, j.lam_fn[l], j.lam_row[l], i), 0.0f);
      for (int p = 0; p < j.lam_order[l]; ++p) f = f * inv_eps;
      LAMs[l * N + i] = f;
    }
    __syncwarp();

    // ---- 2. FP32 Householder QR in registers
    float a[MR][N];
#pragma unroll
    for (int i = 0; i < MR; ++i)
#pragma unroll
      for (int c = 0; c < N; ++c) a[i][c] = Bs[c * LD + lane + 32 * i].h;
    qr_columns<MR, N>(a, TAUs, lane, std::make_integer_sequence<int, N>{});
    // stage R, 1/r_ii; conditioning of the factor
    float rmax = 0.0f, rmin = 3.0e38f;
#pragma unroll
    for (int i = 0; i < MR; ++i) {
      const int r = lane + 32 * i;
      if (r < N) {
#pragma unroll
        for (int c = 0; c < N; ++c) Rs[r * RS + c] = (c >= r) ? a[i][c] : 0.0f;
        float d = 0.0f;
#pragma unroll
        for (int c = 0; c < N; ++c)
          if (c == r) d = a[i][c];
        IDs[r] = 1.0f / d;
        rmax = fmaxf(rmax, fabsf(d));
        rmin = fminf(rmin, fabsf(d));
      }
    }
    rmax = wmax(rmax);
    rmin = -wmax(-rmin);
    __syncwarp();
    const bool ill = !(rmin * 1.0e6f >= rmax) || !(rmin > 0.0f);

    // ---- 3. initial FP32 solve: y0 = R^{-T} lambda, s0 = Q [y0; 0], y = R^{-1} y0
    float w[L][NT];
    float z[L][MR];
#pragma unroll
    for (int l = 0; l < L; ++l)
#pragma unroll
      for (int tt = 0; tt < NT; ++tt) {
        const int p = lane + 32 * tt;
        w[l][tt] = (p < N) ? LAMs[l * N + p].h : 0.0f;
      }
    solve_rt_lanes<N, L>(Rs, RS, IDs, w, lane);
#pragma unroll
    for (int l = 0; l < L; ++l)
#pragma unroll
      for (int i = 0; i < MR; ++i) {
        const int r = lane + 32 * i;
        z[l][i] = (i < NT && r < N) ? w[l][i < NT ? i : 0] : 0.0f;
      }
    apply_q_regs<MR, N, L, true>(a, TAUs, z, lane);
    solve_r_lanes<N, L>(Rs, RS, IDs, w, lane);
#pragma unroll
    for (int l = 0; l < L; ++l) {
#pragma unroll
      for (int i = 0; i < MR; ++i) Ss[l * LD + lane + 32 * i] = ff(z[l][i], 0.0f);
#pragma unroll
      for (int tt = 0; tt < NT; ++tt) {
        const int p = lane + 32 * tt;
        if (p < N) Ys[l * N + p] = ff(w[l][tt], 0.0f);
      }
    }
    __syncwarp();

    // ---- 4. refinement with float-float residuals
    bool conv = false;
    int used = 0;
    float prev = 0.0f;
    for (int iter = 0; iter < j.max_refine && !ill; ++iter) {
      // f = B y - s, lanes over rows
#pragma unroll
      for (int l = 0; l < L; ++l) {
#pragma unroll
        for (int i = 0; i < MR; ++i) {
          const int r = lane + 32 * i;
          Dot2 acc;
          acc.init(-Ss[l * LD + r]);
#pragma unroll
          for (int c = 0; c < N; ++c) acc.add_prod(Bs[c * LD + r], Ys[l * N + c]);
          z[l][i] = __fadd_rn(acc.h, acc.l);
        }
      }
      // g = lambda - B^T s over the L*N (l, c) pairs: whole pairs per lane in
      // full rounds of 32, the remaining pairs split into row blocks so that
      // every lane does about the same number of terms
      {
        const int pairs = L * N, full = pairs / 32, rem = pairs % 32;
        for (int u = 0; u < full; ++u) {
          const int e = u * 32 + lane, l = e / N, c = e % N;
          // four independent compensated chains over interleaved rows (ILP)
          Dot2 acc[4];
          acc[0].init(LAMs[l * N + c]);
          const ff* bc = Bs + c * LD;
          const ff* sl = Ss + l * LD;
#pragma unroll 2
          for (int r = 0; r < ROWS; r += 4) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (r + q < ROWS) acc[q].add_prod(-bc[r + q], sl[r + q]);
          }
          const ff tot = (acc[0].value() + acc[1].value()) + (acc[2].value() + acc[3].value());
          Gs[l * N + c] = __fadd_rn(tot.h, tot.l);
        }
        if (rem) {
          const int nblk = 32 / rem, chunk = (ROWS + nblk - 1) / nblk;
          const int e = full * 32 + lane % rem, blk = lane / rem;
          Dot2 acc;
          if (blk < nblk) {
            const int l = e / N, c = e % N;
            const ff* bc = Bs + c * LD;
            const ff* sl = Ss + l * LD;
            const int r1 = min(ROWS, (blk + 1) * chunk);
            for (int r = blk * chunk; r < r1; ++r) acc.add_prod(-bc[r], sl[r]);
            PARTs[lane] = acc.value();
          }
          __syncwarp();
          if (lane < rem) {
            const int l = e / N, c = e % N;
            ff sum = LAMs[l * N + c];
            for (int b = 0; b < nblk; ++b) sum = sum + PARTs[b * rem + lane];
            Gs[l * N + c] = __fadd_rn(sum.h, sum.l);
          }
        }
      }
      __syncwarp();
      // d = Q^T f ; a = R^{-T} g ; dy = R^{-1} (a - d_1) ; ds = Q [a; d_2]
      apply_q_regs<MR, N, L, false>(a, TAUs, z, lane);
#pragma unroll
      for (int l = 0; l < L; ++l)
#pragma unroll
        for (int tt = 0; tt < NT; ++tt) {
          const int p = lane + 32 * tt;
          w[l][tt] = (p < N) ? Gs[l * N + p] : 0.0f;
        }
      solve_rt_lanes<N, L>(Rs, RS, IDs, w, lane);
      float dyv[L][NT];
#pragma unroll
      for (int l = 0; l < L; ++l)
#pragma unroll
        for (int tt = 0; tt < NT; ++tt) {
          const int p = lane + 32 * tt;
          // rows r < N of z sit in the same lane/slot as entry p = r
          dyv[l][tt] = (p < N) ? w[l][tt] - z[l][tt < MR ? tt : 0] : 0.0f;
          if (p < N && tt < MR) z[l][tt < MR ? tt : 0] = w[l][tt];
        }
      solve_r_lanes<N, L>(Rs, RS, IDs, dyv, lane);
      apply_q_regs<MR, N, L, true>(a, TAUs, z, lane);
      float dmax = 0.0f, smax = 0.0f;
#pragma unroll
      for (int l = 0; l < L; ++l) {
#pragma unroll
        for (int i = 0; i < MR; ++i) {
          const int r = lane + 32 * i;
          const ff s1 = add_f(Ss[l * LD + r], z[l][i]);
          Ss[l * LD + r] = s1;
          dmax = fmaxf(dmax, fabsf(z[l][i]));
          smax = fmaxf(smax, fabsf(s1.h));
        }
#pragma unroll
        for (int tt = 0; tt < NT; ++tt) {
          const int p = lane + 32 * tt;
          if (p < N) Ys[l * N + p] = add_f(Ys[l * N + p], dyv[l][tt]);
        }
      }
      dmax = wmax(dmax);
      smax = wmax(smax);
      __syncwarp();
      used = iter + 1;
      // error left after this correction ~ |ds| times the contraction factor,
      // estimated by the relative size of the correction (first iteration) or
      // by the ratio of successive corrections (later ones)
      const float rho = (iter == 0) ? dmax / fmaxf(smax, 1e-37f) : dmax / fmaxf(prev, 1e-37f);
      const float est = dmax * fminf(1.0f, rho);
      conv = est <= tolf * smax;
      prev = dmax;
      if (conv) break;
    }
    if (!conv) {
      if (lane == 0) {
        const int slot = atomicAdd(j.fb_count, 1);
        j.fb_items[slot] = (int32_t)to;
        j.status[to] = ill ? GMLS_T_ILL_CONDITIONED : GMLS_T_REFINE_NOT_CONVERGED;
      }
      continue;
    }

    // ---- 5. store w = sqrt(W) s (FP64) in [row][neighbour][component]
    for (int f = 0; f < j.nout; ++f) {
      const int R = j.out_rows[f], C = j.out_ncomp[f], src = j.out_src[f];
      double* wo = j.out_w[f] + o0 * (int64_t)R * C;
      const int per_row = k * C;
      const bool div_scalar = (j.out_fn[f] == GMLS_F_DIV) && (KIND == GMLS_BASIS_SCALAR);
      const float sgn = (float)j.out_sign[f];
      for (int rr = 0; rr < R; ++rr) {
        for (int e = lane; e < per_row; e += 32) {
          double val = 0.0;
          if (src >= 0) {
            if (div_scalar) {
              const int q = e / C, c = e % C;
              const ff s = Ss[(src + c) * LD + q] * SWs[q];
              val = to_double(s);
            } else {
              const ff s = Ss[(src + rr) * LD + e] * SWs[e];
              val = to_double(ff(sgn * s.h, sgn * s.l));
            }
          }
          wo[(int64_t)rr * per_row + e] = val;
        }
      }
    }
    if (j.beta)
      for (int l = lane; l < L; l += 32) j.beta[to * L + l] = 0.0;
    if (lane == 0) {
      j.status[to] = st;
      if (j.iters) j.iters[to] = (uint8_t)used;
    }
    __syncwarp();
  }
}

// ----------------------------------------------------------------- dispatch
struct FastEntry {
  int kind, dim, deg, mr, L;
  const void* fn;
  size_t (*bytes)(int L);
};

#define GMLS_FAST(KIND, D, DEG, MR, L)                                                                                \
  FastEntry {                                                                                                          \
    KIND, D, DEG, MR, L, (const void*)stencil_fast_kernel<KIND, D, DEG, MR, L>,                                        \
        &FastLay<MR, gmls_gen::basis_size(KIND, D, DEG)>::bytes                                                        \
  }

}  // namespace gmls
