// stencil_dfx.cuh -- divergence-free GMLS stencils through a factored QR.
// (kernel template; instantiations and dispatch in dfx.cu)
//
// Sec. 2.2 of the paper builds the divergence-free reconstruction on a basis
// of pi^div_m = {v in (pi_m)^d : div v = 0}.  Every component of such a field
// is a scalar polynomial of degree <= m, so with the scaled Taylor monomials
// p_g(xi) = xi^g / g! (Eq. basis-functions-3d) the weighted basis matrix of a
// target factors exactly as
//
//     B[(j, c), i] = sum_g A[j, g] C[(c, g), i],   A = diag(sqrt(W)) P_scalar,
//
// A being the k x Q scalar Taylor tile of degree m (Q = C(m + d, d)) and C a
// constant 0 / +-1 matrix.  The basis used here (any basis of the span gives
// the same stencils) is, with d/dxi_k p_g = p_{g - e_k}:
//
//     phi_{c,g} = e_c p_g - e_0 p_{g - e_c + e_0}    c = 1..d-1, |g| <= m
//                 (second term only when g_c >= 1), div phi = p_{g-e_c} - p_{g-e_c} = 0;
//     phi_{0,g} = e_0 p_g                            g_0 = 0.
//
// That is (d - 1) Q + #{g : g_0 = 0} functions: 9 / 14 / 20 in 2D and 26 / 50
// in 3D for m = 2 / 3 / 4, the dimension of pi^div_m.
//
// Least squares through two QR factorisations (FP32, one warp per target):
//   1. A = Q_A R_A (Householder, the tile in registers);
//   2. G = (I_d (x) R_A) C, rows ordered (components 1..d-1 | component 0),
//      columns (phi_{1,.} .. phi_{d-1,.} | phi_{0,.}).  Its top (d - 1) Q rows
//      are diag(R_A, .., R_A) (upper triangular, zero in the phi_0 columns);
//      only the Q bottom rows need eliminating: column j < (d-1) Q by a
//      reflector on (top row j, bottom rows), the last columns by a dense QR
//      of what is left of the bottom block;
//   3. B = (I (x) Q_A) Q_G R_G is a QR factorisation of B, so R_G is its R
//      factor and Q_B = (I (x) Q_A) Q_G.
// For the 240 x 50 systems of the 3D degree-3 basis this is about 0.17 MFLOP
// of factorisation instead of 1.12 MFLOP for a QR of B.
//
// Solve and refinement: y0 = R^-1 R^-T lambda (FP32), then one Bjorck step on
// the augmented system [[I, B], [B^T, 0]] [s; -y] = [0; lambda^T] starting
// from s0 = B y0 evaluated in float-float, so that f = B y0 - s0 = 0 and the
// correction needs a single application of Q_B:
//   g = lambda - B^T s0 (float-float),  delta = R^-T g,  ds = Q_B [delta; 0].
// s0 = B y0 carries an error of order kappa u_32 (as Q_B [R^-T lambda; 0]
// would) and the step contracts it by about kappa u_32.  B y0 and B^T s0 go
// through the factored form -- u = C y0, s0_(l,c,j) = A_j . u_(l,c);
// v_(l,c) = A^T s0_(l,c), B^T s0 = C^T v -- 2 k Q d L compensated products
// instead of 2 k d n L.  Targets whose correction misses the tolerance, or
// whose factor is ill-conditioned, go to the FP64 redo list.
#pragma once
#include <cuda_runtime.h>

#include <utility>

#include "stencil_fast.cuh"

namespace gmls {

// ------------------------------------------------------------ basis tables
// Scalar Taylor monomials of degree <= M, in the order of the generated
// evaluators (degree ascending; within a degree g_x descending, then g_y).
template <int D, int M>
struct DfxMono {
  static constexpr int Q = D == 2 ? (M + 1) * (M + 2) / 2 : (M + 1) * (M + 2) * (M + 3) / 6;
  int e[Q][3];
  constexpr DfxMono() : e() {
    int i = 0;
    for (int s = 0; s <= M; ++s) {
      if (D == 2) {
        for (int gx = s; gx >= 0; --gx) {
          e[i][0] = gx;
          e[i][1] = s - gx;
          e[i][2] = 0;
          ++i;
        }
      } else {
        for (int gx = s; gx >= 0; --gx)
          for (int gy = s - gx; gy >= 0; --gy) {
            e[i][0] = gx;
            e[i][1] = gy;
            e[i][2] = s - gx - gy;
            ++i;
          }
      }
    }
  }
  constexpr int index(int a, int b, int c) const {
    for (int i = 0; i < Q; ++i)
      if (e[i][0] == a && e[i][1] == b && e[i][2] == c) return i;
    return -1;
  }
};

template <int D, int M>
struct DfxDims {
  static constexpr int Q = DfxMono<D, M>::Q;
  static constexpr int NTOP = (D - 1) * Q;                                  // phi_{c,g}, c >= 1
  static constexpr int N0 = D == 2 ? M + 1 : (M + 1) * (M + 2) / 2;        // phi_{0,g}, g_0 = 0
  static constexpr int N = NTOP + N0;
  static constexpr int L = D;   // solve rows: the vector Laplacian, one per component
  static constexpr int LC = L * D;
};

// Lookup tables with run-time indices (a kernel parameter: constant bank).
//   src[i]:    column i < NTOP (phi_{c,g}): monomial g - e_c + e_0, or -1;
//              column i >= NTOP (phi_{0,g}): monomial g;
//   fidx[g]:   g_0 = 0: position of phi_{0,g} among the phi_0 columns, else -1;
//   ush[c][g]: c >= 1, g_0 >= 1: monomial g + e_c - e_0 (whose phi_{c,.}
//              puts -p_g into component 0), else -1;
//   lam[l][i]: vector Laplacian row l on basis function i, times eps^2.
struct DfxTab {
  int8_t src[64];
  int8_t fidx[32];
  int8_t ush[3][32];
  int8_t lam[3][64];
};

template <int D, int M>
DfxTab make_dfx_tab() {
  constexpr DfxMono<D, M> mo{};
  using Dm = DfxDims<D, M>;
  DfxTab t;
  for (auto& v : t.src) v = -1;
  for (auto& v : t.fidx) v = -1;
  for (auto& r : t.ush)
    for (auto& v : r) v = -1;
  for (auto& r : t.lam)
    for (auto& v : r) v = 0;
  auto is2 = [&](int g) {  // g = 2 e_k for some k
    int two = 0, zero = 0;
    for (int q = 0; q < 3; ++q) {
      two += mo.e[g][q] == 2;
      zero += mo.e[g][q] == 0;
    }
    return two == 1 && zero == 2;
  };
  int f = 0;
  for (int g = 0; g < Dm::Q; ++g)
    if (mo.e[g][0] == 0) {
      t.fidx[g] = (int8_t)f;
      t.src[Dm::NTOP + f] = (int8_t)g;
      if (is2(g)) t.lam[0][Dm::NTOP + f] += 1;
      ++f;
    }
  for (int c = 1; c < D; ++c)
    for (int g = 0; g < Dm::Q; ++g) {
      const int i = (c - 1) * Dm::Q + g;
      int e[3] = {mo.e[g][0], mo.e[g][1], mo.e[g][2]};
      if (is2(g)) t.lam[c][i] += 1;
      if (e[c] >= 1) {
        e[c] -= 1;
        e[0] += 1;
        const int s = mo.index(e[0], e[1], e[2]);
        t.src[i] = (int8_t)s;
        t.ush[c][s] = (int8_t)g;
        if (is2(s)) t.lam[0][i] -= 1;
      }
    }
  return t;
}

// Shared memory of one warp (one target in flight).  KS: neighbour capacity.
// The float-float tile A and the factors of G are never needed at the same
// time: A while the basis is evaluated (phase A) and while the refinement
// forms s0 = A u and v = A^T s0 (D); the factors during the QR (B), the FP32
// solve (C) and the correction (E).  Both live in the first region; the one
// not in use waits in the warp's slot of a global scratch (written once and
// read once, it stays in L2).  s0 is formed HG (l, c) pairs at a time in a
// small buffer and kept in the slot, as is sqrt(W): the lane that stores
// them is the lane that reads them back.  A target of the 3D degree-3 basis
// holds about 16 KB of shared memory instead of 30 KB.
template <int D, int M, int KS>
struct DfxLay {
  using Dm = DfxDims<D, M>;
  static constexpr int Q = Dm::Q, N = Dm::N, NTOP = Dm::NTOP, N0 = Dm::N0, L = Dm::L, LC = Dm::LC;
  static constexpr int LDA = KS + 1;  // odd: rows of different columns in different banks
  static constexpr int QV = (Q + 3) & ~3;  // row stride of the reflector blocks: 16-byte rows
  static constexpr size_t al16(size_t v) { return (v + 15) & ~size_t(15); }
  // the factor block (offsets within the first region)
  static constexpr size_t RG = 0;                                             // float [N(N+1)/2] R_G, rows packed
  static constexpr size_t IDG = al16(RG + sizeof(float) * N * (N + 1) / 2);  // float [N] 1 / r_ii
  static constexpr size_t V1 = al16(IDG + sizeof(float) * N);                // float [NTOP][QV] stage-1 reflectors
  static constexpr size_t V2 = al16(V1 + sizeof(float) * NTOP * QV);         // float [N0][QV] stage-2 reflectors
  static constexpr size_t TAUG = al16(V2 + sizeof(float) * N0 * QV);         // float [N]
  static constexpr size_t TAUA = al16(TAUG + sizeof(float) * N);             // float [Q]
  static constexpr size_t FAC = al16(TAUA + sizeof(float) * Q);              // bytes of the factor block
  static constexpr size_t ABYTES = al16(sizeof(ff) * Q * LDA);               // ff [Q][LDA] A = sqrt(W) P
  static constexpr size_t AFF = 0;
  static constexpr int HG = LC % 3 == 0 ? 3 : 2;            // (l, c) pairs of s0 formed together
  static constexpr size_t S = ABYTES > FAC ? ABYTES : FAC;  // ff [HG][LDA] a group of s0 (R_A, then y0, before it)
  static constexpr size_t UV = al16(S + sizeof(ff) * HG * LDA);              // ff [LC][Q] u = C y0, then v = A^T s0
  static constexpr size_t BYTES = al16(UV + sizeof(ff) * LC * Q);
  // global scratch of one warp: A, the factor block, s0 ff [LC][LDA], sqrt(W) ff [LDA]
  static constexpr size_t S0BYTES = al16(sizeof(ff) * LC * LDA), SWBYTES = al16(sizeof(ff) * LDA);
  static constexpr size_t GF = ABYTES;
  static constexpr size_t GS = GF + FAC;
  static constexpr size_t GW = GS + S0BYTES;
  static constexpr size_t SLOT = (GW + SWBYTES + 255) & ~size_t(255);
  // s0 and sqrt(W) back for the store (end of phase E, when the factor
  // block, the s0 buffer and u / v are no longer needed)
  static constexpr size_t FS0 = 0, FSW = S0BYTES;
  static_assert(S0BYTES + SWBYTES <= BYTES, "s0 and sqrt(W) fit in the warp's shared memory");
  static_assert(LC % HG == 0, "(l, c) pairs in groups");
  static_assert(sizeof(float) * Q * (Q + 1) / 2 <= sizeof(ff) * HG * LDA, "R_A must fit in the s buffer");
  static_assert(sizeof(float) * L * N <= sizeof(ff) * HG * LDA, "y0 must fit in the s buffer");
  static_assert(D <= HG, "the offsets (ff [D][LDA]) must fit in the s buffer");
};

// copy of a 16-byte-aligned block by the 32 lanes of a warp, global side
// cached in L2 only; every lane moves the same vectors in both directions
template <size_t BYTES>
__device__ __forceinline__ void dfx_park(float4* __restrict__ g, const float4* __restrict__ sm, int lane) {
  static_assert(BYTES % 16 == 0, "whole vectors");
#pragma unroll 4
  for (int e = lane; e < (int)(BYTES / 16); e += 32) __stcg(g + e, sm[e]);
}
template <size_t BYTES>
__device__ __forceinline__ void dfx_unpark(float4* __restrict__ sm, const float4* __restrict__ g, int lane) {
  static_assert(BYTES % 16 == 0, "whole vectors");
#pragma unroll 4
  for (int e = lane; e < (int)(BYTES / 16); e += 32) sm[e] = __ldcg(g + e);
}

// x[sl] += v / x[sl] for a run-time slot index (static register indices)
template <int S>
__device__ __forceinline__ void dfx_add_slot(float (&x)[S], int sl, float v) {
#pragma unroll
  for (int i = 0; i < S; ++i)
    if (i == sl) x[i] += v;
}
template <int S>
__device__ __forceinline__ float dfx_get_slot(const float (&x)[S], int sl) {
  float v = x[0];
#pragma unroll
  for (int i = 1; i < S; ++i)
    if (i == sl) v = x[i];
  return v;
}

// z <- Q_A^T z (rev false) or Q_A z (rev true) for V row-distributed vectors
// (row lane + 32 t in z[q][t]); reflector k is column k of the register tile
// below the diagonal (v_k[k] = 1).  The V dot products of a reflector are
// all-reduced together (recursive halving).  One copy of the code serves both
// directions: step s takes column s or Q - 1 - s by a select (the kernel is
// large enough for instruction fetch to matter).
template <int MR, int Q, int V>
__device__ __forceinline__ void dfx_apply_qa(const float (&a)[MR][Q], const float* tau, float (&z)[V][MR], int lane,
                                             unsigned mask, bool rev) {
#pragma unroll
  for (int s = 0; s < Q; ++s) {
    const int k = rev ? Q - 1 - s : s;
    const float tk = tau[k];
    float v[MR];
#pragma unroll
    for (int i = 0; i < MR; ++i) {
      const int r = lane + 32 * i;
      const float ak = rev ? a[i][Q - 1 - s] : a[i][s];
      v[i] = (r > k) ? ak : (r == k ? 1.0f : 0.0f);
    }
    float d[V];
#pragma unroll
    for (int q = 0; q < V; ++q) {
      d[q] = 0.0f;
#pragma unroll
      for (int i = 0; i < MR; ++i) d[q] = fmaf(v[i], z[q][i], d[q]);
    }
    allreduce_tail<32, V, 0>(d, lane, mask);
#pragma unroll
    for (int q = 0; q < V; ++q) {
      const float dq = d[q] * tk;
#pragma unroll
      for (int i = 0; i < MR; ++i) z[q][i] = fmaf(-dq, v[i], z[q][i]);
    }
  }
}

// Triangular solves with the packed rows of R in shared memory (R(i, p) at
// rpk<N>(i, p)), right-hand sides in the solve layout (entry p at lane p % 32,
// slot p / 32), loops over the pivot rolled: w <- R^-T w (TRANS) or R^-1 w.
template <int N, int L, int NT, bool TRANS>
__device__ __forceinline__ void dfx_solve(const float* Rs, const float* idg, float (&w)[L][NT], int lane,
                                          unsigned mask) {
  // R^T: row i of R (packed from rpk(i, 0)) updates entries p > i;
  // R: column i, entry (p, i) at rpk(p, 0) + i for this lane's rows p
  int pb[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const int p = lane + 32 * t;
    pb[t] = rpk<N>(p < N ? p : N - 1, 0);
  }
#pragma unroll 1
  for (int s = 0; s < N; ++s) {
    const int i = TRANS ? s : N - 1 - s;
    const float inv = idg[i];
    const int src = i & 31, sl = i >> 5;
    const int ri = TRANS ? rpk<N>(i, 0) : 0;
    float yi[L];
#pragma unroll
    for (int l = 0; l < L; ++l) yi[l] = __shfl_sync(mask, dfx_get_slot<NT>(w[l], sl), src) * inv;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int p = lane + 32 * t;
      const bool upd = TRANS ? (p > i && p < N) : (p < i);
      const float r = upd ? Rs[TRANS ? ri + p : pb[t] + i] : 0.0f;
#pragma unroll
      for (int l = 0; l < L; ++l) {
        if (p == i) w[l][t] = yi[l];
        w[l][t] = fmaf(-r, yi[l], w[l][t]);
      }
    }
  }
}

// z <- Q_G^T z (FWD) or Q_G z in the row space of G: top rows p < NTOP at
// lane p % 32, slot p / 32 of zt; bottom rows r < Q at lane r of zb.
// Stage-1 reflector jst acts on (top row jst, bottom rows) with vector
// (1, V1[jst][.]); stage-2 reflector j2 on the bottom rows with V2[j2][.]
// (rows QV floats apart)
// (one at row j2, zero above).
template <int L, int TS, int Q, int QV, int NTOP, int N0, bool FWD>
__device__ __forceinline__ void dfx_apply_qg(float (&zt)[L][TS], float (&zb)[L], const float* V1, const float* V2,
                                             const float* taug, int lane, unsigned mask) {
  auto stage1 = [&](int jst) {
    const float v = lane < Q ? V1[jst * QV + lane] : 0.0f;
    const float tk = taug[jst];
    const int own = jst & 31, sl = jst >> 5;
    float d[L];
#pragma unroll
    for (int l = 0; l < L; ++l) d[l] = fmaf(v, zb[l], lane == own ? dfx_get_slot<TS>(zt[l], sl) : 0.0f);
    allreduce_tail<32, L, 0>(d, lane, mask);
#pragma unroll
    for (int l = 0; l < L; ++l) {
      const float dl = d[l] * tk;
      zb[l] = fmaf(-dl, v, zb[l]);
      if (lane == own) dfx_add_slot<TS>(zt[l], sl, -dl);
    }
  };
  auto stage2 = [&](int j2) {
    const float v = lane < Q ? V2[j2 * QV + lane] : 0.0f;
    const float tk = taug[NTOP + j2];
    float d[L];
#pragma unroll
    for (int l = 0; l < L; ++l) d[l] = v * zb[l];
    allreduce_tail<32, L, 0>(d, lane, mask);
#pragma unroll
    for (int l = 0; l < L; ++l) zb[l] = fmaf(-d[l] * tk, v, zb[l]);
  };
  if (FWD) {
#pragma unroll 1
    for (int jst = 0; jst < NTOP; ++jst) stage1(jst);
#pragma unroll 1
    for (int j2 = 0; j2 < N0; ++j2) stage2(j2);
  } else {
#pragma unroll 1
    for (int j2 = N0 - 1; j2 >= 0; --j2) stage2(j2);
#pragma unroll 1
    for (int jst = NTOP - 1; jst >= 0; --jst) stage1(jst);
  }
}

// v[0..Q) = row[0..Q) in 16-byte loads: a row of a [.][QV] float array
// (QV = Q rounded up to a multiple of 4) at a 16-byte aligned base; the
// padding entries are loaded and dropped
template <int Q>
__device__ __forceinline__ void dfx_load_row(const float* row, float (&v)[Q]) {
  const float4* r4 = reinterpret_cast<const float4*>(row);
#pragma unroll
  for (int i = 0; i < (Q + 3) / 4; ++i) {
    const float4 t = r4[i];
    const float e[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (4 * i + u < Q) v[4 * i + u] = e[u];
  }
}

// Householder reflector of a column held by one lane: alpha the diagonal
// entry, x[r] for r in (lo, Q) the entries below it.  Writes the reflector
// vector (vout[r]: 1 at r == lo when lo >= 0, zero above), tau and beta.
// c + v . x in four interleaved chains
template <int Q>
__device__ __forceinline__ float dfx_dot4(const float (&v)[Q], const float (&x)[Q], float c) {
  float d[4] = {c, 0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int r = 0; r < Q; ++r) d[r & 3] = fmaf(v[r], x[r], d[r & 3]);
  return (d[0] + d[1]) + (d[2] + d[3]);
}

template <int Q>
__device__ __forceinline__ void dfx_reflect(float alpha, const float (&x)[Q], int lo, float* vout, float* tau_out,
                                            float* beta_out) {
  float sg[4] = {0.0f, 0.0f, 0.0f, 0.0f};  // four chains (latency)
#pragma unroll
  for (int r = 0; r < Q; ++r)
    if (r > lo) sg[r & 3] = fmaf(x[r], x[r], sg[r & 3]);
  const float sig = (sg[0] + sg[1]) + (sg[2] + sg[3]);
  float tk = 0.0f, beta = alpha, scale = 0.0f;
  if (sig > 0.0f) {
    const float nrm = sqrtf(fmaf(alpha, alpha, sig));
    beta = alpha >= 0.0f ? -nrm : nrm;
    scale = __fdividef(1.0f, alpha - beta);
    tk = __fdividef(beta - alpha, beta);
  }
#pragma unroll
  for (int r = 0; r < Q; ++r) vout[r] = r > lo ? x[r] * scale : (r == lo ? 1.0f : 0.0f);
  *tau_out = tk;
  *beta_out = beta;
}

// Up to MAXT / 32 warps (targets) per block, each on its own; the bound caps
// the registers so that that many warps fit on an SM: 384 threads (168
// registers) for the 3D degree-3 basis (about 16 KB of shared memory a
// warp), more for the smaller bases (their instantiations in dfx.cu).  The
// warps of a block take consecutive targets (shared neighbours in L1) and
// their scratch slots are adjacent.
template <int D, int M, int MRA, int KS, int MAXT = 384>
__global__ void __launch_bounds__(MAXT, 1) stencil_dfx_kernel(StencilJob j, const DfxTab tab) {
  using Dm = DfxDims<D, M>;
  constexpr int Q = Dm::Q, N = Dm::N, NTOP = Dm::NTOP, N0 = Dm::N0, L = Dm::L, LC = Dm::LC;
  constexpr int NT = (N + 31) / 32;     // slots of an N-vector (solve layout)
  constexpr int TS = (NTOP + 31) / 32;  // slots of the top rows of G
  static_assert(Q <= 32 && N <= 64 && NTOP <= 64 && KS <= 32 * MRA && N0 <= Q, "tile outside this kernel's layout");
  static_assert(N == gmls_gen::basis_size(GMLS_BASIS_DIVFREE, D, M), "dimension of the divergence-free span");
  using Lay = DfxLay<D, M, KS>;
  constexpr int LDA = Lay::LDA, QV = Lay::QV;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const unsigned mask = 0xffffffffu;
  unsigned char* base = smem + (size_t)wid * Lay::BYTES;
  ff* Aff = reinterpret_cast<ff*>(base + Lay::AFF);      // phases A and D (see DfxLay)
  ff* SG = reinterpret_cast<ff*>(base + Lay::S);         // a group of s0 = B y0 (float-float)
  float* RA = reinterpret_cast<float*>(base + Lay::S);   // R_A, packed rows (phase B)
  float* Y0 = reinterpret_cast<float*>(base + Lay::S);   // y0 of pass 0 (FP32; phases C, D)
  ff* UV = reinterpret_cast<ff*>(base + Lay::UV);
  // the factor block: phases B, C and E
  float* RG = reinterpret_cast<float*>(base + Lay::RG);
  float* IDG = reinterpret_cast<float*>(base + Lay::IDG);
  float* V1 = reinterpret_cast<float*>(base + Lay::V1);
  float* V2 = reinterpret_cast<float*>(base + Lay::V2);
  float* TAUG = reinterpret_cast<float*>(base + Lay::TAUG);
  float* TAUA = reinterpret_cast<float*>(base + Lay::TAUA);
  float4* gA = reinterpret_cast<float4*>(j.dscratch + ((size_t)blockIdx.x * wpb + wid) * Lay::SLOT);
  float4* gF = gA + Lay::GF / 16;
  float2* gS = reinterpret_cast<float2*>(gA + Lay::GS / 16);  // s0, ff [LC][LDA]
  float2* gW = reinterpret_cast<float2*>(gA + Lay::GW / 16);  // sqrt(W), ff [LDA]
  const ff* S0F = reinterpret_cast<const ff*>(base + Lay::FS0);  // phase E: s0 (all pairs)
  const ff* SWF = reinterpret_cast<const ff*>(base + Lay::FSW);  // phase E: sqrt(W)
  const int64_t n = j.n;
  const int64_t n_items = j.items ? (int64_t)(*j.n_items) : j.n_tgt;
  const float tolf = (float)j.tol;

  for (int64_t it = (int64_t)blockIdx.x * wpb + wid; it < n_items; it += (int64_t)gridDim.x * wpb) {
    const int64_t to = j.items ? (int64_t)j.items[it] : it;
    const int64_t t = j.tgt[to];
    const int64_t o0 = j.off[to];
    const int k = (int)(j.off[to + 1] - o0);
    uint8_t st = j.nbr_status ? j.nbr_status[to] : 0;
    const bool too_few = (st & GMLS_T_TOO_FEW_NEIGHBOURS) || k <= 0 || !(j.eps[to] > 0.0);
    if (!too_few && (k < Q || k > KS || j.L != L)) {
      // not for this path: the shared-memory FP32 kernel takes it
      if (lane == 0) {
        const int slot = atomicAdd(j.gen_count, 1);
        j.gen_items[slot] = (int32_t)to;
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
        for (int l = lane; l < j.L; l += 32) j.beta[to * j.L + l] = 0.0;
      if (lane == 0) {
        j.status[to] = st;
        if (j.iters) j.iters[to] = 0;
      }
      continue;
    }

    // ---- 1. A = sqrt(W) P (scalar Taylor tile) in float-float, FP32 copy in registers
    const ff eps(j.eps[to]);
    const ff inv_eps = recip(eps);
    const ff ie2 = inv_eps * inv_eps;
    double xt[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int c = 0; c < D; ++c) xt[c] = j.x[c * n + t];
    const int half_p = j.wpow_half;
    // offsets x_j - x_T of this lane's rows into the s0 buffer (the loads of
    // all rows in flight together)
    ff* DX = SG;  // ff [D][LDA]
    {
      double xv[MRA][D];
#pragma unroll
      for (int tt = 0; tt < MRA; ++tt) {
        const int q = lane + 32 * tt;
        const int32_t jj = q < k ? j.idx[o0 + q] : (int32_t)t;
#pragma unroll
        for (int c = 0; c < D; ++c) xv[tt][c] = j.x[c * n + jj];
      }
#pragma unroll
      for (int tt = 0; tt < MRA; ++tt) {
        const int q = lane + 32 * tt;
        if (q < k)
#pragma unroll
          for (int c = 0; c < D; ++c) DX[c * LDA + q] = diff_ff(xv[tt][c], xt[c]);
      }
    }
#pragma unroll 1
    for (int q = lane; q < k; q += 32) {
      ff dx[3], xi[3];
      ff r2(0.f, 0.f);
#pragma unroll
      for (int c = 0; c < D; ++c) {
        dx[c] = DX[c * LDA + q];
        xi[c] = dx[c] * inv_eps;
        r2 = r2 + dx[c] * dx[c];
      }
      const ff u = ff(1.f, 0.f) - sqrt_ff(r2) * inv_eps;
      ff sw(0.f, 0.f);
      if (u.h > 0.0f) {
        sw = u;
        for (int pp = 1; pp < half_p; ++pp) sw = sw * u;
      }
      gmls_gen::BasisEval<GMLS_BASIS_SCALAR, D, M>::template run<ff>(xi, Aff + q, LDA, sw);
      __stcg(gW + q, make_float2(sw.h, sw.l));  // the constant column of A
    }
    __syncwarp(mask);
    float a[MRA][Q];
#pragma unroll
    for (int tt = 0; tt < MRA; ++tt) {
      const int q = lane + 32 * tt;
#pragma unroll
      for (int g = 0; g < Q; ++g) a[tt][g] = q < k ? Aff[g * LDA + q].h : 0.0f;
    }
    // A waits in global memory while the factor block takes its place
    dfx_park<Lay::ABYTES>(gA, reinterpret_cast<const float4*>(Aff), lane);
    __syncwarp(mask);

    // ---- 2. A = Q_A R_A in registers; R_A row r (lane r) packed into RA
    qr_columns<32, MRA, Q>(a, TAUA, lane, mask, std::make_integer_sequence<int, Q>{});
    if (lane < Q) {
#pragma unroll
      for (int c = 0; c < Q; ++c)
        if (c >= lane) RA[rpk<Q>(lane, c)] = a[0][c];
    }
    __syncwarp(mask);

    // ---- 3. G = (I (x) R_A) C: the bottom block (component 0 rows), one
    //         column per lane and slot (column lane + 32 s)
    float xg[NT][Q];
#pragma unroll
    for (int s = 0; s < NT; ++s) {
      const int col = lane + 32 * s;
      const int src = col < N ? (int)tab.src[col] : -1;
      const float sgn = col < NTOP ? -1.0f : 1.0f;
#pragma unroll
      for (int r = 0; r < Q; ++r) {
        xg[s][r] = 0.0f;
        if (src >= r) xg[s][r] = sgn * RA[rpk<Q>(r, src)];  // R_A is upper triangular
      }
    }
    // stage 1: column jst < NTOP against top row jst (R_A row al of block blk)
#pragma unroll 1
    for (int jst = 0; jst < NTOP; ++jst) {
      const int blk = jst / Q, al = jst - blk * Q;
      if (lane == (jst & 31)) {
        float beta, tk;
        const float alpha = RA[rpk<Q>(al, al)];
        if (NT == 1 || jst < 32)
          dfx_reflect<Q>(alpha, xg[0], -1, V1 + jst * QV, &tk, &beta);
        else
          dfx_reflect<Q>(alpha, xg[NT - 1], -1, V1 + jst * QV, &tk, &beta);
        TAUG[jst] = tk;
        RG[rpk<N>(jst, jst)] = beta;
      }
      __syncwarp(mask);
      const float tk = TAUG[jst];
      float v[Q];
      dfx_load_row<Q>(V1 + jst * QV, v);
#pragma unroll
      for (int s = 0; s < NT; ++s) {
        const int col = lane + 32 * s;
        if (col > jst && col < N) {
          const int cb = col / Q, cg = col - cb * Q;
          float tc = 0.0f;  // T[jst][col]: R_A row al within the same block
          if (col < NTOP && cb == blk && cg >= al) tc = RA[rpk<Q>(al, cg)];
          const float dot = dfx_dot4<Q>(v, xg[s], tc) * tk;
          RG[rpk<N>(jst, col)] = tc - dot;
#pragma unroll
          for (int r = 0; r < Q; ++r) xg[s][r] = fmaf(-dot, v[r], xg[s][r]);
        }
      }
      __syncwarp(mask);
    }
    // stage 2: dense QR of the remaining bottom-block columns
#pragma unroll 1
    for (int j2 = 0; j2 < N0; ++j2) {
      const int colk = NTOP + j2;
      if (lane == (colk & 31)) {
        float beta, tk;
        float alpha = 0.0f;
        if (NT == 1 || colk < 32) {
#pragma unroll
          for (int r = 0; r < Q; ++r)
            if (r == j2) alpha = xg[0][r];
          dfx_reflect<Q>(alpha, xg[0], j2, V2 + j2 * QV, &tk, &beta);
        } else {
#pragma unroll
          for (int r = 0; r < Q; ++r)
            if (r == j2) alpha = xg[NT - 1][r];
          dfx_reflect<Q>(alpha, xg[NT - 1], j2, V2 + j2 * QV, &tk, &beta);
        }
        TAUG[colk] = tk;
        RG[rpk<N>(colk, colk)] = beta;
      }
      __syncwarp(mask);
      const float tk = TAUG[colk];
      float v[Q];
      dfx_load_row<Q>(V2 + j2 * QV, v);
#pragma unroll
      for (int s = 0; s < NT; ++s) {
        const int col = lane + 32 * s;
        if (col > colk && col < N) {
          const float dot = dfx_dot4<Q>(v, xg[s], 0.0f) * tk;
          float rrow = 0.0f;
#pragma unroll
          for (int r = 0; r < Q; ++r) {
            xg[s][r] = fmaf(-dot, v[r], xg[s][r]);
            if (r == j2) rrow = xg[s][r];
          }
          RG[rpk<N>(colk, col)] = rrow;
        }
      }
      __syncwarp(mask);
    }
    // 1 / r_ii and the conditioning of the factor
    float rmax = 0.0f, rmin = 3.0e38f;
#pragma unroll
    for (int s = 0; s < NT; ++s) {
      const int p = lane + 32 * s;
      if (p < N) {
        const float d = RG[rpk<N>(p, p)];
        IDG[p] = 1.0f / d;
        rmax = fmaxf(rmax, fabsf(d));
        rmin = fminf(rmin, fabsf(d));
      }
    }
    rmax = wmax<32>(rmax, mask);
    rmin = -wmax<32>(-rmin, mask);
    const bool ill = !(rmin * 1.0e6f >= rmax) || !(rmin > 0.0f);
    __syncwarp(mask);

    // ---- 4. pass 0 (the plain FP32 solve) and one refinement pass.  A
    //         target whose correction misses the tolerance after that pass
    //         (about 2e-4 of the targets of the porous workload) goes on to
    //         the shared-memory FP32 kernel, or to the FP64 kernel when its
    //         factor is ill conditioned; s = s0 + ds is formed only when the
    //         weights are stored.
    auto lam = [&](int l, int i) {  // vector Laplacian row l at basis function i (float-float)
      const int c = tab.lam[l][i];
      return c == 0 ? ff(0.f, 0.f) : mul_f(ie2, (float)c);
    };
    // z = Q_B [dl; 0] for L vectors dl in the solve layout: Q_G in the row
    // space of G, then Q_A on each (l, c) vector (row layout)
    auto apply_qb = [&](const float (&dl)[L][NT], float (&z)[LC][MRA]) {
      float zt[L][TS], zb[L];
#pragma unroll
      for (int l = 0; l < L; ++l) {
#pragma unroll
        for (int s = 0; s < TS; ++s) {
          const int p = lane + 32 * s;
          zt[l][s] = p < NTOP ? dl[l][s < NT ? s : 0] : 0.0f;
        }
        // bottom row r < N0 holds dl[NTOP + r]
        const int p = NTOP + lane;
        const float b0 = __shfl_sync(mask, dl[l][0], p & 31);
        const float b1 = NT > 1 ? __shfl_sync(mask, dl[l][NT - 1], p & 31) : 0.0f;
        zb[l] = lane < N0 ? ((p >> 5) == 0 ? b0 : b1) : 0.0f;
      }
      dfx_apply_qg<L, TS, Q, QV, NTOP, N0, false>(zt, zb, V1, V2, TAUG, lane, mask);
#pragma unroll
      for (int l = 0; l < L; ++l) {
        z[l * D][0] = lane < Q ? zb[l] : 0.0f;
#pragma unroll
        for (int c = 1; c < D; ++c) {
          const int p = (c - 1) * Q + lane;  // top row of (component c, R_A row lane)
          const float s0 = __shfl_sync(mask, zt[l][0], p & 31);
          const float s1 = TS > 1 ? __shfl_sync(mask, zt[l][TS - 1], p & 31) : 0.0f;
          z[l * D + c][0] = lane < Q ? ((p >> 5) == 0 ? s0 : s1) : 0.0f;
        }
#pragma unroll
        for (int c = 0; c < D; ++c)
#pragma unroll
          for (int tt = 1; tt < MRA; ++tt) z[l * D + c][tt] = 0.0f;
      }
      dfx_apply_qa<MRA, Q, LC>(a, TAUA, z, lane, mask, true);
    };

    // pass 0: y0 = R^-1 R^-T lambda (FP32).  The refinement starts from
    // s0 = B y0 evaluated in float-float, so that f = B y0 - s0 = 0 exactly
    // and the Bjorck correction needs one application of Q_B:
    //   g = lambda - B^T s0,  delta = R^-T g,  ds = Q_B [delta; 0].
    // (s0 = B y0 is as accurate as Q_B [R^-T lambda; 0] -- its error is of
    // order kappa u_32 -- and the correction contracts it by about kappa u_32.)
    float w[L][NT];
#pragma unroll
    for (int l = 0; l < L; ++l)
#pragma unroll
      for (int s = 0; s < NT; ++s) {
        const int p = lane + 32 * s;
        w[l][s] = p < N ? lam(l, p).h : 0.0f;
      }
    dfx_solve<N, L, NT, true>(RG, IDG, w, lane, mask);
    dfx_solve<N, L, NT, false>(RG, IDG, w, lane, mask);
#pragma unroll
    for (int l = 0; l < L; ++l)
#pragma unroll
      for (int s = 0; s < NT; ++s) {
        const int p = lane + 32 * s;
        if (p < N) Y0[l * N + p] = w[l][s];
      }
    __syncwarp(mask);

    bool conv = false;
    float z[LC][MRA];
    if (!ill && j.max_refine >= 1) {
      // the factor block out, A back in
      dfx_park<Lay::FAC>(gF, reinterpret_cast<const float4*>(RG), lane);
      __syncwarp(mask);
      dfx_unpark<Lay::ABYTES>(reinterpret_cast<float4*>(Aff), gA, lane);
      // u = C y0 (exact in float-float: sums of at most d FP32 values)
      for (int e = lane; e < LC * Q; e += 32) {
        const int lc = e / Q, g = e - lc * Q, l = lc / D, c = lc - l * D;
        ff uv(0.f, 0.f);
        if (c >= 1) {
          uv = ff(Y0[l * N + (c - 1) * Q + g], 0.f);
        } else if (tab.fidx[g] >= 0) {
          uv = ff(Y0[l * N + NTOP + tab.fidx[g]], 0.f);
        } else {
#pragma unroll
          for (int c2 = 1; c2 < D; ++c2) {
            const int ug = tab.ush[c2][g];
            if (ug >= 0) uv = uv - ff(Y0[l * N + (c2 - 1) * Q + ug], 0.f);
          }
        }
        UV[e] = uv;
      }
      __syncwarp(mask);
      // per group of HG (l, c) pairs: s0 = B y0, row (l, c, j) = A_j . u_(l,c)
      // (compensated; into the buffer and the slot), then v_(l,c) = A^T s0_(l,c)
      // over it (four interleaved compensated chains per entry), in place of u
      constexpr int HG = Lay::HG;
#pragma unroll 1
      for (int lg = 0; lg < LC; lg += HG) {
#pragma unroll 1
        for (int q = lane; q < k; q += 32) {
          Dot2 acc[HG];
#pragma unroll
          for (int g = 0; g < Q; ++g) {
            const ff ag = Aff[g * LDA + q];
#pragma unroll
            for (int h = 0; h < HG; ++h) acc[h].add_prod(ag, UV[(lg + h) * Q + g]);
          }
#pragma unroll
          for (int h = 0; h < HG; ++h) {
            const ff sv = acc[h].value();
            SG[h * LDA + q] = sv;
            __stcg(gS + (lg + h) * LDA + q, make_float2(sv.h, sv.l));
          }
        }
        __syncwarp(mask);
        for (int e = lane; e < HG * Q; e += 32) {
          const int h = e / Q, g = e - h * Q;
          const ff* ag = Aff + g * LDA;
          const ff* sl = SG + h * LDA;
          Dot2 c4[4];
          int q = 0;
          for (; q + 3 < k; q += 4) {
#pragma unroll
            for (int i = 0; i < 4; ++i) c4[i].add_prod(ag[q + i], sl[q + i]);
          }
          for (; q < k; ++q) c4[0].add_prod(ag[q], sl[q]);
          UV[(lg + h) * Q + g] = (c4[0].value() + c4[1].value()) + (c4[2].value() + c4[3].value());
        }
        __syncwarp(mask);
      }
      // A is no longer needed: the factor block back
      dfx_unpark<Lay::FAC>(reinterpret_cast<float4*>(RG), gF, lane);
      __syncwarp(mask);
      // g = lambda - C^T v in the solve layout
#pragma unroll
      for (int l = 0; l < L; ++l)
#pragma unroll
        for (int s = 0; s < NT; ++s) {
          const int i = lane + 32 * s;
          float gv = 0.0f;
          if (i < N) {
            ff ct(0.f, 0.f);
            if (i < NTOP) ct = UV[(l * D + 1 + i / Q) * Q + i % Q];
            const int src = tab.src[i];
            if (src >= 0) {
              const ff v0 = UV[(l * D) * Q + src];
              ct = i < NTOP ? ct - v0 : ct + v0;
            }
            const ff gg = lam(l, i) - ct;
            gv = __fadd_rn(gg.h, gg.l);
          }
          w[l][s] = gv;
        }
      dfx_solve<N, L, NT, true>(RG, IDG, w, lane, mask);  // delta = R^-T g
      apply_qb(w, z);                                      // ds = Q_B [delta; 0]
      // s0 and sqrt(W) back from the slot in one batch of loads, in place
      // of the factor block
      __syncwarp(mask);
      dfx_unpark<Lay::S0BYTES>(reinterpret_cast<float4*>(base + Lay::FS0), reinterpret_cast<const float4*>(gS), lane);
      dfx_unpark<Lay::SWBYTES>(reinterpret_cast<float4*>(base + Lay::FSW), reinterpret_cast<const float4*>(gW), lane);
      __syncwarp(mask);
      // error left ~ |ds| times the contraction factor, estimated by the
      // relative size of the correction
      float dmax = 0.0f, smax = 0.0f;
#pragma unroll
      for (int lc = 0; lc < LC; ++lc)
#pragma unroll
        for (int tt = 0; tt < MRA; ++tt) {
          const int q = lane + 32 * tt;
          if (q < k) {
            const float s0h = S0F[lc * LDA + q].h;
            dmax = fmaxf(dmax, fabsf(z[lc][tt]));
            smax = fmaxf(smax, fabsf(s0h + z[lc][tt]));
          }
        }
      dmax = wmax<32>(dmax, mask);
      smax = wmax<32>(smax, mask);
      const float rho = dmax / fmaxf(smax, 1e-37f);
      conv = dmax * fminf(1.0f, rho) <= tolf * smax;
    }
    if (!conv) {
      if (lane == 0) {
        if (!ill && j.max_refine > 1) {
          // well conditioned, but one pass was not enough: the
          // shared-memory FP32 kernel, which refines further (its own
          // misses go to the FP64 kernel)
          const int slot = atomicAdd(j.gen_count, 1);
          j.gen_items[slot] = (int32_t)to;
          j.status[to] = 0;
        } else {
          const int slot = atomicAdd(j.fb_count, 1);
          j.fb_items[slot] = (int32_t)to;
          j.status[to] = ill ? GMLS_T_ILL_CONDITIONED : GMLS_T_REFINE_NOT_CONVERGED;
        }
      }
      __syncwarp(mask);
      continue;
    }

    // ---- 5. w = sqrt(W) (s0 + ds) (FP64) in [row][neighbour][component],
    //         from the row layout
    for (int fo = 0; fo < j.nout; ++fo) {
      const int R = j.out_rows[fo], C = j.out_ncomp[fo], src = j.out_src[fo];
      double* wo = j.out_w[fo] + o0 * (int64_t)R * C;
      if (src < 0) {
        for (int e = lane; e < R * k * C; e += 32) wo[e] = 0.0;
        continue;
      }
      const float sgn = (float)j.out_sign[fo];
#pragma unroll
      for (int tt = 0; tt < MRA; ++tt) {
        const int q = lane + 32 * tt;
        if (q < k) {
          const ff swq = SWF[q];
#pragma unroll
          for (int l = 0; l < L; ++l)
#pragma unroll
            for (int c = 0; c < D; ++c) {
              const int rr = l - src;
              if (rr >= 0 && rr < R && c < C) {
                const ff wv = add_f(S0F[(l * D + c) * LDA + q], z[l * D + c][tt]) * swq;
                __stcs(wo + ((int64_t)rr * k + q) * C + c, to_double(ff(sgn * wv.h, sgn * wv.l)));
              }
            }
        }
      }
    }
    if (j.beta)
      for (int l = lane; l < j.L; l += 32) j.beta[to * j.L + l] = 0.0;
    if (lane == 0) {
      j.status[to] = st;
      if (j.iters) j.iters[to] = 1;
    }
    __syncwarp(mask);
  }
}

// ----------------------------------------------------------------- dispatch
struct DfxEntry {
  int dim, deg, mra, ks;
  const void* fn;
  size_t bytes;  // shared memory per warp
  size_t slot;   // global scratch per warp
  DfxTab (*tab)();
};

#define GMLS_DFX(D, M, MRA, KS, MAXT)                                                                        \
  DfxEntry {                                                                                                 \
    D, M, MRA, KS, (const void*)stencil_dfx_kernel<D, M, MRA, KS, MAXT>, DfxLay<D, M, KS>::BYTES,            \
        DfxLay<D, M, KS>::SLOT, &make_dfx_tab<D, M>                                                          \
  }

}  // namespace gmls
