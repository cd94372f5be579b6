// Field solves as dense DFT / sine-transform GEMMs on the 5th-generation tensor
// cores (tcgen05), operands staged by TMA into 128-byte-swizzled shared
// memory, accumulators in TMEM, 3-term split precision:
//   a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi,   a_hi = r(a), a_lo = r(a - a_hi),
// accumulated in FP32, with r the rounding to TF32 (kind::tf32, operands kept
// as fp32) or, for the open-boundary solve only, to BF16 (kind::f16 with bf16
// operands, half the operand bytes; 8 + 8 significant bits per split value).
//
// The convolution of Hockney's method (zero-padded doubled grid, Mx = 2nx,
// My = 2ny) with the centred-difference field kernels Dx, Dy (spectra i Sx,
// i Sy) factorises into four real GEMMs C = A B^T (both operands K-major):
//   P1  R1T[c][j]  = B1[c][i] q[j][i]             row DFT of the real charge,
//       c <= nx: Re F1(j, p=c); c = nx+p: Im F1(j, p)           (half spectrum)
//   P2A F[r][p]    = W2f[r][(re|im, j)] B2[p][(re|im, j)]   column DFT over j,
//       r < My: Re F(k=r, p), r = My+k: Im F; epilogue H_f = i S_f F
//   P2B G[r][(f,p)] = W2i[r][(re|im, k)] B3[(f,p)][(re|im, k)]  inverse column
//       DFT, kept for j' < ny: r < ny: Re G_f(j', p), r = ny+j': Im G_f
//   P3  E[(f,j)][i] = A3[(f,j)][(re|im, p)] B4[i][(re|im, p)]   Hermitian
//       inverse row DFT with weights 1 (p = 0, nx) or 2 and 1/(Mx My).
// Supported: nx = ny in {64, 128, 256} (M tiles of 128 rows).
//
// The conducting pipe of Sec. IV-B (walls on the outer nodes) uses the same
// kernel with four more phases and the real sine matrix S of the m interior
// nodes (padded to mp, whole 128-row tiles), F the right-hand side
// -2 pi q / (hx hy) on the interior:
//   D1  T1[p][j]  = S[p][i] F[j][i]               row sine transform
//   D2  UT[p][q]  = (S[q][j] T1[p][j]) / lambda_pq column transform, division
//   D3  T3[(f,j)][p] = [S; Cy][(f,j)][q] UT[p][q]  inverse columns, f = 1: d/dy
//   D4  [(f,j)][(h,i)] = T3[(f,j)][p] [S; Cx][(h,i)][p] x 4/(m+1)^2:
//       (0,0) potential, (0,1) Ex, (1,0) Ey at interior node (i+1, j+1)
// with Cx, Cy the centred differences of the sine modes (cosine series).
//
// Stacked grids (slices, bunches of a batch) extend the data operand, so one
// launch per phase covers them.  Tile width (N columns per CTA), split-K
// cluster size and pipeline depth are chosen per phase by timing the
// candidates when a grid is created.
#include <cooperative_groups.h>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "sc_internal.cuh"

namespace sc {

namespace {

// Operand element of the split products.  A K chunk is one 128-byte swizzle
// row either way: 32 fp32 (TF32) or 64 bf16 elements; each MMA takes 32 bytes
// of K (8 TF32 or 16 BF16 elements), four per chunk.
enum Elem { E_TF32 = 0, E_BF16 = 1 };
template <int EL>
struct Op;
template <>
struct Op<E_TF32> {
  using T = float;
  static constexpr int KC = 32;
};
template <>
struct Op<E_BF16> {
  using T = __nv_bfloat16;
  static constexpr int KC = 64;
};
__host__ __device__ constexpr int kc_of(int el) { return el == E_BF16 ? 64 : 32; }
constexpr int TM = 128;         // rows per MMA / M tile
constexpr int kThreads = 128;   // 4 warps: TMA producer, MMA issuer, TMEM owner, all do the epilogue
constexpr long long kWaitCycles = 4000000000LL;  // bounded mbarrier waits (~2 s of SM clock), then error + bail out

// P1..P3: open-boundary convolution; D1..D4: conducting-pipe sine transforms
enum Phase { P1 = 0, P2A = 1, P2B = 2, P3 = 3, D1 = 4, D2 = 5, D3 = 6, D4 = 7 };

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false once kWaitCycles SM clocks have passed (the caller records the error).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)tm), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
template <int EL>
__device__ __forceinline__ void mma_split(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if (EL == E_BF16)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 32 lanes x 16 consecutive 32-bit columns: this thread gets its lane's 16 values.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r[c]);
}

// UMMA shared-memory descriptor, K-major, 128-byte swizzle: start address,
// leading offset 1 (unused for this layout), stride 1024 B between 8-row
// groups, descriptor version 1, layout SWIZZLE_128B.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
// hi/lo split of a value for the 3-term products (TF32 values kept as fp32, or bf16)
__device__ __forceinline__ void split(float x, float& hi, float& lo) {
  hi = tf32_round(x);
  lo = tf32_round(x - hi);
}
__device__ __forceinline__ void split(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// Split four consecutive values and store hi and lo as one vector each (16 B
// of fp32, or 8 B of bf16; the destinations are aligned to 4 elements).
__device__ __forceinline__ void store_split4(float* dh, float* dl, const float* v) {
  float h[4], l[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) split(v[u], h[u], l[u]);
  *(float4*)dh = make_float4(h[0], h[1], h[2], h[3]);
  *(float4*)dl = make_float4(l[0], l[1], l[2], l[3]);
}
__device__ __forceinline__ void store_split4(__nv_bfloat16* dh, __nv_bfloat16* dl, const float* v) {
  __align__(8) __nv_bfloat16 h[4], l[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) split(v[u], h[u], l[u]);
  *(uint2*)dh = *(const uint2*)h;
  *(uint2*)dl = *(const uint2*)l;
}

// byte offset of the element at byte kb < 128 of row r in a K-major SW128 tile of 128-byte rows
__device__ __forceinline__ uint32_t sw128_offset_bytes(int r, int kb) {
  return (uint32_t)(r * 128 + ((((kb >> 4) ^ (r & 7)) << 4) | (kb & 15)));
}

struct GemmArgs {
  CUtensorMap tA_hi, tA_lo, tB_hi, tB_lo;  // tB_* unused for P1
  int k_chunks;   // K / (elements per K chunk)
  int m_tiles;    // M tiles (TM rows each) of the whole, possibly stacked, GEMM
  int n_tiles;    // N tiles (NT columns each)
  int n_total;    // valid columns (the last tile may run past them)
  int nx, ny, My, Npad;
  // P1: charge input (stacked grids back to back: row n of the GEMM's N is Q row n)
  const unsigned long long* Q;
  float scale;
  const float* stack_scale;  // per stacked grid (bunches of a batch), or NULL: scale
  float qfac;                // D1: extra factor of the charge (-2 pi / (hx hy)); P1: 1
  // P2A: charge grid to clear for the next deposit (NULL: leave it)
  unsigned long long* Qzero;
  long long qcells;
  // outputs / epilogue inputs
  void *out_hi, *out_lo;   // next phase's operand (P1: B2, P2A: B3, P2B: A3), fp32 or bf16
  int out_ld;              // its row length (K of the next phase)
  long long out_slice;     // its elements per stacked grid
  const float *Sx, *Sy;    // P2A: spectra [Npad][My]
  float2* E;               // P3: fields, float32 (Ex, Ey) per node
  long long e_slice;       // P3: nodes per stacked grid
  int* err;                // set to 1 when a bounded wait ran out
  // conducting pipe (D phases): m interior nodes per axis, mp = m padded to whole M tiles
  int m, mp;
  const float* inv_lam;    // D2: 1 / lambda at (q, p), [mp][mp], 0 in the padding
  float norm;              // D4: 4 / (m+1)^2
  float* phi;              // D4: potential [stacked grid][ny][nx] (walls stay 0)
  // failure-detection test: announce the data operand's copies to the stage
  // barriers without issuing them, so every bounded wait runs out
  int drop_data_loads;
};

// Which operand is a constant DFT matrix (loadable before the grid dependency
// resolves) and which is the previous kernel's output.
template <int PH>
struct Roles {
  static constexpr bool CONST_A = (PH != P3 && PH != D4);
  static constexpr bool TMA_B = (PH != P1 && PH != D1);
};

template <int PH, int NT, int STAGES_>
struct Smem {
  static constexpr int A_TILE = TM * 128;  // bytes of one 128-row x 32-element tile
  static constexpr int B_TILE = NT * 128;
  static constexpr int STAGE = 2 * A_TILE + (Roles<PH>::TMA_B ? 2 * B_TILE : 0);
  static constexpr int STAGES = STAGES_;
  static constexpr int B_RESIDENT_MAX_CHUNKS = 8;  // P1: charge tiles for K up to 256
  static constexpr int RESIDENT = (PH == P1 || PH == D1) ? 2 * B_RESIDENT_MAX_CHUNKS * B_TILE : 0;
  static constexpr int BYTES = STAGES * STAGE + RESIDENT + 1024 /*align slack*/;
  static_assert(BYTES <= 227 * 1024, "shared memory of one CTA");
};
// split-K reduction buffer after the stages and resident tiles: SK slots of this
// CTA's NT / SK columns for all TM rows, float32
template <int SK, int NT>
constexpr int red_bytes() {
  return SK > 1 ? TM * NT * 4 : 0;
}

// Instruction descriptor: D f32, A = B = tf32 (kind::tf32: format 2) or bf16
// (kind::f16: format 1), both K-major, M = 128, N = NT.
template <int NT, int EL>
__host__ __device__ constexpr uint32_t idesc() {
  return (1u << 4) | ((EL == E_BF16 ? 1u : 2u) << 7) | ((EL == E_BF16 ? 1u : 2u) << 10) |
         ((uint32_t)(NT >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

namespace cg = cooperative_groups;
__device__ __forceinline__ void prefetch_map(const CUtensorMap* m) {
  asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)m) : "memory");
}

// One cluster of SK CTAs: a 128-row x NT-column tile of C = A B^T, the K
// chunks split evenly across the SK CTAs; each accumulates its three split
// products in TMEM, the partial tiles are summed through distributed shared
// memory and each CTA finishes NT/SK of the columns.  Stacked grids (slices,
// bunches of a batch) extend the data operand: their rows follow one another,
// so one launch covers all of them; tiles are ordered so that consecutive
// CTAs share the data operand's tile (the constant one stays in L2).
template <int PH, int SK, int NT, int STAGES, int EL>
__global__ void __launch_bounds__(kThreads, 1) dft_gemm(const __grid_constant__ GemmArgs g) {
  using L = Smem<PH, NT, STAGES>;
  using R = Roles<PH>;
  static_assert(L::BYTES + red_bytes<SK, NT>() <= 227 * 1024, "shared memory of one CTA");
  using T = typename Op<EL>::T;
  constexpr int KC = Op<EL>::KC;
  T* const out_hi = (T*)g.out_hi;
  T* const out_lo = (T*)g.out_lo;
  // Narrow tiles (NT <= 32), where an MMA's time goes mostly to reading its A slice:
  // accumulators [0, 2 NT) = a_hi [b_hi | b_lo] (one MMA of width 2 NT over the two B
  // tiles, which lie back to back in shared memory: the A slice is read once for both
  // products) and [2 NT, 3 NT) = a_lo b_hi, summed by the epilogue.  Wider tiles: the
  // three products in one accumulator of NT columns (a few CTAs' allocations then fit
  // an SM's tensor memory, so the next phase's CTAs allocate while this one runs).
  constexpr bool FUSE = NT <= 32;
  constexpr int TMEM_COLS = FUSE ? (3 * NT <= 64 ? 64 : 128) : (NT < 32 ? 32 : NT);
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[L::STAGES], empty_bar[L::STAGES], accum_bar;
  __shared__ uint32_t tmem_base_s;
  __shared__ volatile int abort_s;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rank = (SK > 1) ? (int)cg::this_cluster().block_rank() : 0;
  const int tile = blockIdx.x / SK;
  // data operand outer: B (P1, P2A, P2B) or A (P3)
  const int mb = R::CONST_A ? tile % g.m_tiles : tile / g.n_tiles;
  const int nb = R::CONST_A ? tile / g.m_tiles : tile % g.n_tiles;
  const int n0 = nb * NT, a_row = mb * TM;
  unsigned char* stage_base = smem;
  unsigned char* resident = smem + L::STAGES * L::STAGE;
  const int kpc = g.k_chunks / SK, kc0 = rank * kpc;  // this CTA's K chunks: kc0 .. kc0+kpc-1
  const int pre = kpc < L::STAGES ? kpc : L::STAGES;

  auto load_a = [&](int lk, int st) {
    unsigned char* sb = stage_base + st * L::STAGE;
    tma_load_2d(sb, &g.tA_hi, &full_bar[st], (kc0 + lk) * KC, a_row);
    tma_load_2d(sb + L::A_TILE, &g.tA_lo, &full_bar[st], (kc0 + lk) * KC, a_row);
  };
  auto load_b = [&](int lk, int st) {
    unsigned char* bb = stage_base + st * L::STAGE + 2 * L::A_TILE;
    tma_load_2d(bb, &g.tB_hi, &full_bar[st], (kc0 + lk) * KC, n0);
    tma_load_2d(bb + L::B_TILE, &g.tB_lo, &full_bar[st], (kc0 + lk) * KC, n0);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < L::STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&accum_bar, 1);
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    prefetch_map(&g.tA_hi);
    prefetch_map(&g.tA_lo);
    if (R::TMA_B) {
      prefetch_map(&g.tB_hi);
      prefetch_map(&g.tB_lo);
    }
  }
  if (warp == 2) tmem_alloc(&tmem_base_s, TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;

  // P2A: the spectra of this thread's row for the epilogue's first column chunk, loaded
  // now (constants): left to the epilogue, their latency sat on the solve's critical path
  constexpr int CW = NT / SK;             // columns finished by this CTA
  constexpr int CH = CW < 16 ? CW : 16;   // columns per epilogue chunk
  const int c0 = rank * CW;
  float pre_sx[CH], pre_sy[CH];
  if (PH == P2A) {
    const int rr = a_row + threadIdx.x, kr = rr < g.My ? rr : rr - g.My;
    const int nb = n0 + c0, s0 = nb / g.Npad, q0 = nb - s0 * g.Npad;
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const bool wrap = q0 + u >= g.Npad;  // CH <= 16 <= Npad: at most one grid boundary
      const int pq = q0 + u - (wrap ? g.Npad : 0);
      const bool in = nb + u < g.n_total;
      pre_sx[u] = in ? __ldg(g.Sx + (size_t)pq * g.My + kr) : 0.f;
      pre_sy[u] = in ? __ldg(g.Sy + (size_t)pq * g.My + kr) : 0.f;
    }
  }

  // constant operand of the first stages: independent of the previous kernel
  if (threadIdx.x == 0) {
    for (int kc = 0; kc < pre; ++kc) {
      mbar_expect_tx(&full_bar[kc], (uint32_t)L::STAGE);
      if (R::CONST_A)
        load_a(kc, kc);
      else
        load_b(kc, kc);
    }
  }
  pdl_wait();
  if ((PH == P2A || PH == D2) && g.Qzero) {
    // every reader of the charge (the row transform) has finished: clear it for the next deposit
    for (long long c = (long long)blockIdx.x * kThreads + threadIdx.x; c < g.qcells;
         c += (long long)gridDim.x * kThreads)
      g.Qzero[c] = 0ull;
  }
  if (PH == P1) {
    // B operand = normalised charge rows n0 .. n0+NT-1 (NT divides ny: one stacked grid per
    // tile), this CTA's K columns kcol0 .. kcol0+kcols-1 (all nx without split-K), split
    // hi/lo, swizzled; 16-byte loads, issued in groups of 8.
    const int kcol0 = kc0 * KC, kcols = kpc * KC;
    const int hx = kcols >> 1;  // column pairs per row
    const int pairs = NT * hx;
    const longlong2* q2 = (const longlong2*)(g.Q + (size_t)n0 * g.nx + kcol0);
    const int row2 = g.nx >> 1;  // a charge row in pairs
    const float qscale = g.qfac * (g.stack_scale ? g.stack_scale[n0 / g.ny] : g.scale);
    constexpr int G = 8;
    // pair e = (row r, columns kcol0 + 2c, +1) with r = e / hx: this thread's pairs are
    // e = threadIdx.x + m kThreads, walked with a running (r, c) -- no division per pair
    const int step_r = kThreads / hx, step_c = kThreads - step_r * hx;
    int pr = threadIdx.x / hx, pc = threadIdx.x - pr * hx;
    for (int e0 = threadIdx.x; e0 < pairs; e0 += G * kThreads) {
      longlong2 v[G];
      {
        int lr = pr, lc = pc;
#pragma unroll
        for (int u = 0; u < G; ++u) {
          const int e = e0 + u * kThreads;
          v[u] = (e < pairs) ? q2[lr * row2 + lc] : make_longlong2(0, 0);
          lr += step_r;
          lc += step_c;
          if (lc >= hx) {
            lc -= hx;
            ++lr;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < G; ++u) {
        const int e = e0 + u * kThreads;
        const int r = pr;
        const int i0 = 2 * pc;
        pr += step_r;
        pc += step_c;
        if (pc >= hx) {
          pc -= hx;
          ++pr;
        }
        if (e < pairs) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const unsigned long long qi = (unsigned long long)(h ? v[u].y : v[u].x);
            const int i = kcol0 + i0 + h;
            // uint64 -> float through its 32-bit halves (no FP64 instruction)
            const float qv =
                fmaf(__uint2float_rn((unsigned)(qi >> 32)), 4294967296.f, __uint2float_rn((unsigned)qi)) * qscale;
            T hi, lo;
            split(qv, hi, lo);
            const int kc = i / KC, kb = (i % KC) * (int)sizeof(T);
            *(T*)(resident + (2 * kc) * L::B_TILE + sw128_offset_bytes(r, kb)) = hi;
            *(T*)(resident + (2 * kc + 1) * L::B_TILE + sw128_offset_bytes(r, kb)) = lo;
          }
        }
      }
    }
    fence_proxy_async();
  }
  if (PH == D1) {
    // B operand = interior charge rows of the pipe grid: GEMM row n0 + r = (stacked grid s, interior
    // row j) <- charge row j+1, K = i <- column i+1, zero beyond the m interior nodes (mp divides
    // by NT: one stacked grid per tile); scaled to the right-hand side -2 pi q / (hx hy).
    const int s0 = n0 / g.mp, j0 = n0 - s0 * g.mp;
    const unsigned long long* q = g.Q + (size_t)s0 * g.nx * g.ny;
    const float qscale = g.qfac * (g.stack_scale ? g.stack_scale[s0] : g.scale);
    const int elems = NT * g.mp;
    constexpr int G = 8;
    for (int e0 = threadIdx.x; e0 < elems; e0 += G * kThreads) {
      unsigned long long v[G];
#pragma unroll
      for (int u = 0; u < G; ++u) {
        const int e = e0 + u * kThreads;
        const int r = e / g.mp, i = e - r * g.mp, j = j0 + r;
        v[u] = (e < elems && i < g.m && j < g.m) ? q[(size_t)(j + 1) * g.nx + (i + 1)] : 0ull;
      }
#pragma unroll
      for (int u = 0; u < G; ++u) {
        const int e = e0 + u * kThreads;
        if (e < elems) {
          const int r = e / g.mp, i = e - r * g.mp;
          const float qv =
              fmaf(__uint2float_rn((unsigned)(v[u] >> 32)), 4294967296.f, __uint2float_rn((unsigned)v[u])) * qscale;
          T hi, lo;
          split(qv, hi, lo);
          const int kc = i / KC, kb = (i % KC) * (int)sizeof(T);
          *(T*)(resident + (2 * kc) * L::B_TILE + sw128_offset_bytes(r, kb)) = hi;
          *(T*)(resident + (2 * kc + 1) * L::B_TILE + sw128_offset_bytes(r, kb)) = lo;
        }
      }
    }
    fence_proxy_async();
  }
  __syncthreads();

  if (warp == 0 && lane == 0) {
    // ---- TMA producer: the data operand of the prefetched stages, then whole stages
    for (int kc = 0; kc < pre && !g.drop_data_loads; ++kc) {
      if (R::CONST_A) {
        if (R::TMA_B) load_b(kc, kc);
      } else {
        load_a(kc, kc);
      }
    }
    for (int kc = pre; kc < kpc; ++kc) {
      const int st = kc % L::STAGES;
      if (!mbar_wait(&empty_bar[st], ((kc / L::STAGES) - 1) & 1)) {
        abort_s = 1;
        break;
      }
      mbar_expect_tx(&full_bar[st], (uint32_t)L::STAGE);
      load_a(kc, st);
      if (R::TMA_B) load_b(kc, st);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    for (int kc = 0; kc < kpc; ++kc) {
      const int st = kc % L::STAGES;
      if (!mbar_wait(&full_bar[st], (kc / L::STAGES) & 1)) {
        abort_s = 1;
        break;
      }
      tc_fence_after();
      unsigned char* sb = stage_base + st * L::STAGE;
      const unsigned char* bh =
          (PH == P1 || PH == D1) ? resident + (2 * (kc0 + kc)) * L::B_TILE : sb + 2 * L::A_TILE;
      const uint64_t dbh = desc_sw128(smem_u32(bh));  // b_hi; b_lo follows at bh + B_TILE
      const uint64_t dah = desc_sw128(smem_u32(sb)), dal = desc_sw128(smem_u32(sb + L::A_TILE));
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t o = (uint64_t)(kk * 2);  // 32 bytes per K step, in 16-byte units
        const uint32_t acc = (kc > 0 || kk > 0) ? 1u : 0u;
        if (FUSE) {
          mma_split<EL>(tmem, dah + o, dbh + o, idesc<2 * NT, EL>(), acc);       // a_hi b_hi | a_hi b_lo
          mma_split<EL>(tmem + 2 * NT, dal + o, dbh + o, idesc<NT, EL>(), acc);  // a_lo b_hi
        } else {
          const uint64_t dbl = desc_sw128(smem_u32(bh + L::B_TILE));
          mma_split<EL>(tmem, dah + o, dbh + o, idesc<NT, EL>(), acc);
          mma_split<EL>(tmem, dah + o, dbl + o, idesc<NT, EL>(), 1u);
          mma_split<EL>(tmem, dal + o, dbh + o, idesc<NT, EL>(), 1u);
        }
      }
      mma_commit(&empty_bar[st]);
    }
    // always: the accumulator barrier completes once every MMA issued so far has
    // finished, so TMEM is never freed under an MMA in flight
    mma_commit(&accum_bar);
  }
  __syncwarp();
  pdl_allow();

  // ---- epilogue: all four warps; warp w owns TMEM lanes / tile rows 32w .. 32w+31
  // warp-uniform decisions (tcgen05.ld is a warp-collective instruction)
  const bool have = __all_sync(0xffffffffu, mbar_wait(&accum_bar, 0));
  if ((!have || abort_s) && threadIdx.x == 0) atomicExch(g.err, 1);
  tc_fence_after();
  const int t = warp * 32 + lane;
  const int r = a_row + t;  // row of C
  const bool ok = __all_sync(0xffffffffu, have && !abort_s);
  static_assert(CW % 4 == 0, "whole float4 column groups");
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  // 16 columns of C from column ta: the three split products' accumulators summed
  auto tmem_ld_c16 = [&](uint32_t ta, float (&v)[16]) {
    tmem_ld16(ta, v);
    if (FUSE) {
      float b[16], c[16];
      tmem_ld16(ta + NT, b);
      tmem_ld16(ta + 2 * NT, c);
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = (v[q] + b[q]) + c[q];
    }
  };

  // Finish columns cb .. cb+CH-1 of the tile (values in acc) for this phase.
  auto finish = [&](const float* acc, int cb) {
    if (PH == P1) {
      // row c of R1T: Re F1(j, p = c) for c <= nx, Im F1(j, p = c - nx) above; column = charge row
      const int p = (r <= g.nx) ? r : r - g.nx;
      const int half = (r <= g.nx) ? 0 : 1;
      const int slice = n0 / g.ny, j = n0 - slice * g.ny + cb;
      const size_t ob = (size_t)slice * g.out_slice + (size_t)p * g.out_ld + half * g.ny + j;
#pragma unroll
      for (int q4 = 0; q4 < CH / 4; ++q4) store_split4(out_hi + ob + 4 * q4, out_lo + ob + 4 * q4, acc + 4 * q4);
    } else if (PH == P2A) {
      // row r < My: Re F(k = r, p) -> Im H_f = S_f Re F (column My + k of B3)
      // row r >= My: Im F(k = r - My, p) -> Re H_f = -S_f Im F (column k)
      const bool re = r < g.My;
      const int k = re ? r : r - g.My;
      const int col = re ? g.My + k : k;
      const float sgn = re ? 1.f : -1.f;
      // stacked column n = n0 + cb + u: grid n / Npad, p = n % Npad (one division per
      // chunk); the first chunk's spectra were loaded before the main loop, the
      // others' are loaded here, all before the stores (which could alias them)
      const int sl0 = (n0 + cb) / g.Npad, p0 = n0 + cb - sl0 * g.Npad;
      float sx[CH], sy[CH];
      int sl[CH], pp[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int n = n0 + cb + u;
        const bool wrap = p0 + u >= g.Npad;
        sl[u] = sl0 + (wrap ? 1 : 0);
        pp[u] = p0 + u - (wrap ? g.Npad : 0);
        const bool in = n < g.n_total;
        sx[u] = cb == c0 ? pre_sx[u] : in ? __ldg(g.Sx + (size_t)pp[u] * g.My + k) : 0.f;
        sy[u] = cb == c0 ? pre_sy[u] : in ? __ldg(g.Sy + (size_t)pp[u] * g.My + k) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        if (n0 + cb + u >= g.n_total) continue;
        const float f = sgn * acc[u];
        const size_t base = (size_t)sl[u] * g.out_slice;
        const size_t rx = base + (size_t)pp[u] * g.out_ld + col;
        const size_t ry = base + (size_t)(g.Npad + pp[u]) * g.out_ld + col;
        split(sx[u] * f, out_hi[rx], out_lo[rx]);
        split(sy[u] * f, out_hi[ry], out_lo[ry]);
      }
    } else if (PH == P2B) {
      // row r: part (Re G, Im G) = r / ny at j' = r % ny; stacked column n: grid n / (2 Npad),
      // field f and p within it (4-column groups never straddle: Npad is a multiple of 16)
      const int part = r / g.ny, jr = r % g.ny;
#pragma unroll
      for (int q4 = 0; q4 < CH / 4; ++q4) {
        const int n = n0 + cb + 4 * q4;
        if (n >= g.n_total) continue;
        const int slice = n / (2 * g.Npad), rem = n - slice * 2 * g.Npad;
        const int f = rem / g.Npad, p = rem - f * g.Npad;
        const size_t o = (size_t)slice * g.out_slice + (size_t)(f * g.ny + jr) * g.out_ld + part * g.Npad + p;
        store_split4(out_hi + o, out_lo + o, acc + 4 * q4);
      }
    } else if (PH == P3) {
      // stacked row r: grid r / (2 ny); within it field f = (r % 2ny) / ny (Ex, Ey) at j;
      // columns i = n0 + cb + u; float32 (Ex, Ey) pairs
      const int slice = r / (2 * g.ny), rr = r - slice * 2 * g.ny;
      const int f = rr / g.ny, j = rr % g.ny;
      float* e = (float*)g.E + 2 * ((size_t)slice * g.e_slice + (size_t)j * g.nx + n0 + cb) + f;
#pragma unroll
      for (int u = 0; u < CH; ++u) e[2 * u] = acc[u];
    } else if (PH == D1 || PH == D3) {
      // D1: row p, columns (s, j) -> T1[s][p][j];  D3: row j, columns (s, p) -> T3[s][j][p]
      // (one stacked grid per tile, consecutive columns contiguous)
      const int s0 = n0 / g.mp, c = n0 - s0 * g.mp + cb;
      const size_t ob = (size_t)s0 * g.out_slice + (size_t)r * g.out_ld + c;
#pragma unroll
      for (int q4 = 0; q4 < CH / 4; ++q4) store_split4(out_hi + ob + 4 * q4, out_lo + ob + 4 * q4, acc + 4 * q4);
    } else if (PH == D2) {
      // row q, columns (s, p): U = W / lambda_pq, stored transposed UT[s][p][q] (K = q of D3)
      float il[CH];
      int sl[CH], pp[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int n = n0 + cb + u;
        sl[u] = n / g.mp;
        pp[u] = n - sl[u] * g.mp;
        il[u] = n < g.n_total ? __ldg(g.inv_lam + (size_t)r * g.mp + pp[u]) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        if (n0 + cb + u >= g.n_total) continue;
        const size_t o = (size_t)sl[u] * g.out_slice + (size_t)pp[u] * g.out_ld + r;
        split(acc[u] * il[u], out_hi[o], out_lo[o]);
      }
    } else {
      // D4: stacked row (s, f, j) with f = 0: T3 (potential part), 1: its y-derivative; columns
      // (h, i) with h = 0: S, 1: the x-derivative matrix (one h per tile).  Blocks (0,0) phi,
      // (0,1) Ex, (1,0) Ey at interior node (i+1, j+1) of grid s; (1,1) is not used.
      const int s0 = r / (2 * g.mp), rr = r - s0 * 2 * g.mp;
      const int f = rr / g.mp, j = rr - f * g.mp;
      const int hblk = n0 / g.mp, i0 = n0 - hblk * g.mp + cb;
      if (j < g.m && !(f == 1 && hblk == 1)) {
        const size_t node = (size_t)s0 * g.e_slice + (size_t)(j + 1) * g.nx + 1;
        float* out = (f == 0 && hblk == 0) ? g.phi + node : (float*)g.E + 2 * node + (f == 0 ? 0 : 1);
        const int step = (f == 0 && hblk == 0) ? 1 : 2;
#pragma unroll
        for (int u = 0; u < CH; ++u) {
          const int i = i0 + u;
          if (i < g.m) out[(size_t)step * i] = acc[u] * g.norm;
        }
      }
    }
  };

  if (SK > 1) {
    // Partial tiles summed across the cluster: each CTA stores the columns rank r
    // finishes (CW of them) into rank r's reduction buffer (shared memory of its
    // own, not the stages), slot = the storing CTA's rank; one cluster barrier
    // (release / acquire) makes them visible, and each CTA sums its slots locally.
    // No CTA touches another's shared memory after the barrier, so none waits for
    // the others before leaving.  After a timed-out wait nothing is stored, the
    // barrier is still taken (every CTA of the cluster reaches it), and the error
    // word marks the results invalid.
    cg::cluster_group cl = cg::this_cluster();
    float4* red = (float4*)(smem + L::STAGES * L::STAGE + L::RESIDENT);  // [SK][kThreads][CW / 4]
    if (have) {
#pragma unroll
      for (int c16 = 0; c16 < NT / 16; ++c16) {
        float v[16];
        tmem_ld_c16(trow + c16 * 16, v);
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
          const int col = c16 * 16 + 4 * q4, owner = col / CW, cc = col - owner * CW;
          float4* dst = owner == rank ? red : cl.map_shared_rank(red, owner);
          dst[(rank * kThreads + t) * (CW / 4) + cc / 4] =
              make_float4(v[4 * q4], v[4 * q4 + 1], v[4 * q4 + 2], v[4 * q4 + 3]);
        }
      }
    }
    cl.sync();
#pragma unroll
    for (int cb = c0; cb < c0 + CW; cb += CH) {
      float acc[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u) acc[u] = 0.f;
#pragma unroll
      for (int q = 0; q < SK; ++q) {
#pragma unroll
        for (int q4 = 0; q4 < CH / 4; ++q4) {
          const float4 w = red[(q * kThreads + t) * (CW / 4) + (cb - c0) / 4 + q4];
          acc[4 * q4] += w.x;
          acc[4 * q4 + 1] += w.y;
          acc[4 * q4 + 2] += w.z;
          acc[4 * q4 + 3] += w.w;
        }
      }
      if (ok) finish(acc, cb);
    }
  } else if (ok) {
#pragma unroll
    for (int c16 = 0; c16 < NT / 16; ++c16) {
      float acc[16];
      tmem_ld_c16(trow + c16 * 16, acc);
      finish(acc, c16 * 16);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    // after a timed-out wait, issued MMAs get a second bounded wait to finish
    // before their tensor memory is released
    if (!have) (void)__all_sync(0xffffffffu, mbar_wait(&accum_bar, 0));
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// Fields of the conducting-pipe form on the walls (the interior comes from the
// derivative GEMMs): centred differences with the odd extension across the
// walls reduce to the first interior potential over h for the normal
// component; the tangential component vanishes (phi = 0 along a wall).
__global__ void pipe_walls32(const float* __restrict__ phi, int nx, int ny, int nstack, float inv_hx, float inv_hy,
                             float2* __restrict__ E) {
  pdl_wait();
  const int per = 2 * nx + 2 * (ny - 2);  // perimeter nodes of one grid
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nstack * per; c += gridDim.x * blockDim.x) {
    const int s = c / per, k = c - s * per;
    int i, j;
    if (k < nx) {
      i = k;
      j = 0;
    } else if (k < 2 * nx) {
      i = k - nx;
      j = ny - 1;
    } else if (k < 2 * nx + ny - 2) {
      i = 0;
      j = k - 2 * nx + 1;
    } else {
      i = nx - 1;
      j = k - 2 * nx - (ny - 2) + 1;
    }
    const float* p = phi + (size_t)s * nx * ny;
    float ex = 0.f, ey = 0.f;
    if (i == 0 && j > 0 && j < ny - 1) ex = -p[(size_t)j * nx + 1] * inv_hx;
    if (i == nx - 1 && j > 0 && j < ny - 1) ex = p[(size_t)j * nx + nx - 2] * inv_hx;
    if (j == 0 && i > 0 && i < nx - 1) ey = -p[(size_t)nx + i] * inv_hy;
    if (j == ny - 1 && i > 0 && i < nx - 1) ey = p[(size_t)(ny - 2) * nx + i] * inv_hy;
    E[(size_t)s * nx * ny + (size_t)j * nx + i] = make_float2(ex, ey);
  }
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

sc_status get_encoder() {
  if (g_encode) return SC_OK;
  cudaDriverEntryPointQueryResult q;
  void* fn = nullptr;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
    return set_error(SC_ERR_CUDA, "cuTensorMapEncodeTiled entry point not available");
  g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  return SC_OK;
}

// 2-D row-major [rows][cols] tensor map of fp32 (TF32 operands) or bf16
// elements with boxes of one K chunk (128 bytes) x box_rows, 128-byte swizzle.
sc_status make_map(CUtensorMap* tm, const void* base, int rows, int cols, int box_rows, int el) {
  const size_t esz = el == E_BF16 ? 2 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * esz};
  cuuint32_t box[2] = {(cuuint32_t)kc_of(el), (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = g_encode(tm, el == E_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                        (void*)base, dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(SC_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  return SC_OK;
}

float tf32_host(float x) {
  uint32_t b;
  std::memcpy(&b, &x, 4);
  b = (b + 0x1000u) & ~0x1FFFu;  // round to nearest, ties away, to 10 mantissa bits
  float r;
  std::memcpy(&r, &b, 4);
  return r;
}

// bf16 bits of a float, rounded to nearest, ties to even (finite inputs)
uint16_t bf16_bits_host(float x) {
  uint32_t b;
  std::memcpy(&b, &x, 4);
  b += 0x7FFFu + ((b >> 16) & 1u);
  return (uint16_t)(b >> 16);
}
float bf16_value_host(uint16_t h) {
  const uint32_t b = (uint32_t)h << 16;
  float r;
  std::memcpy(&r, &b, 4);
  return r;
}

// hi/lo split of constant matrices on the host, as raw operand bytes (fp32 or bf16)
void split_host(const std::vector<double>& a, int el, std::vector<unsigned char>& hi, std::vector<unsigned char>& lo) {
  const size_t esz = el == E_BF16 ? 2 : 4;
  hi.resize(a.size() * esz);
  lo.resize(a.size() * esz);
  for (size_t i = 0; i < a.size(); ++i) {
    if (el == E_BF16) {
      const uint16_t h = bf16_bits_host((float)a[i]);
      const uint16_t l = bf16_bits_host((float)(a[i] - (double)bf16_value_host(h)));
      std::memcpy(&hi[i * 2], &h, 2);
      std::memcpy(&lo[i * 2], &l, 2);
    } else {
      const float h = tf32_host((float)a[i]);
      const float l = tf32_host((float)(a[i] - (double)h));
      std::memcpy(&hi[i * 4], &h, 4);
      std::memcpy(&lo[i * 4], &l, 4);
    }
  }
}

struct Mat {
  void* hi = nullptr;
  void* lo = nullptr;
  int rows = 0, cols = 0;
};

}  // namespace

// One phase of the solve as launched: kernel variant, its arguments, its grid.
struct PhaseRun {
  int variant = -1;  // index into the phase's candidate list
  int el = 0;        // operand element (E_TF32 or E_BF16)
  GemmArgs a;
  int grid = 0;
};

struct Tf32Plan {
  int el = E_TF32;           // operand element: E_TF32 or E_BF16 (open boundary only)
  int Mx, My, Npad;
  Mat B1, W2f, W2i, B4;      // constants
  Mat B2, B3, A3;            // intermediates (next phase operands)
  float *Sx, *Sy;            // [Npad][My]
  int K3;                    // row length of A3 and B4 (2 Npad rounded up to whole split-K chunks)
  int* err;
  // conducting pipe (phases D1..D4): sine matrix, intermediates, 1/lambda, potential
  bool pipe = false;
  int m = 0, mp = 0;
  Mat S, SCy, SCx, T1, UT, T3;  // S; [S; Cy] (rows of D3); [S; Cx] (rows of D4's B)
  float* inv_lam = nullptr;  // [mp][mp]
  float* phi = nullptr;      // [nstack][ny][nx]
  PhaseRun run[4];           // the chain's four phases (P1..P3 or D1..D4)
  int drop_data_loads = 0;   // failure-detection test (sc_test_bounded_waits)
  float tuned_us[4];         // time of the chosen variant when tuned (0: forced)
  int base() const { return pipe ? D1 : P1; }
};

namespace {

sc_status upload(Mat& m, const std::vector<double>& v, int rows, int cols, int el) {
  std::vector<unsigned char> hi, lo;
  split_host(v, el, hi, lo);
  m.rows = rows;
  m.cols = cols;
  SC_CUDA(cudaMalloc(&m.hi, hi.size()));
  SC_CUDA(cudaMalloc(&m.lo, lo.size()));
  SC_CUDA(cudaMemcpy(m.hi, hi.data(), hi.size(), cudaMemcpyHostToDevice));
  SC_CUDA(cudaMemcpy(m.lo, lo.data(), lo.size(), cudaMemcpyHostToDevice));
  return SC_OK;
}

sc_status alloc_zero(Mat& m, int rows, int cols, int el) {
  const size_t bytes = (size_t)rows * cols * (el == E_BF16 ? 2 : 4);
  m.rows = rows;
  m.cols = cols;
  SC_CUDA(cudaMalloc(&m.hi, bytes));
  SC_CUDA(cudaMalloc(&m.lo, bytes));
  SC_CUDA(cudaMemset(m.hi, 0, bytes));
  SC_CUDA(cudaMemset(m.lo, 0, bytes));
  return SC_OK;
}

void free_mat(Mat& m) {
  cudaFree(m.hi);
  cudaFree(m.lo);
  m = Mat{};
}

// ------------------------------------------------------------------ kernel variants
struct Variant {
  int sk, nt, stages, smem;
  const void* fn;
};

template <int PH, int SK, int NT, int ST, int EL = E_TF32>
Variant variant() {
  return Variant{SK, NT, ST, Smem<PH, NT, ST>::BYTES + red_bytes<SK, NT>(), (const void*)dft_gemm<PH, SK, NT, ST, EL>};
}

// Candidates per phase (split-K cluster size SK, tile width NT, pipeline
// stages), timed against each other when a grid is created.  Wide tiles load
// each constant-operand tile once for many columns (stacked grids); narrow,
// K-split tiles give a single small grid enough CTAs.
const std::vector<Variant>& variants(int ph, int el = E_TF32) {
  static const std::vector<Variant> v[8] = {
      {variant<P1, 1, 16, 4>(), variant<P1, 1, 32, 4>(), variant<P1, 1, 64, 2>(), variant<P1, 2, 16, 4>()},
      {variant<P2A, 2, 16, 5>(), variant<P2A, 1, 32, 4>(), variant<P2A, 2, 32, 4>(), variant<P2A, 1, 64, 4>(),
       variant<P2A, 1, 128, 3>()},
      {variant<P2B, 4, 16, 5>(), variant<P2B, 2, 32, 4>(), variant<P2B, 1, 64, 4>(), variant<P2B, 2, 64, 4>(),
       variant<P2B, 1, 128, 3>()},
      {variant<P3, 2, 16, 5>(), variant<P3, 1, 32, 4>(), variant<P3, 2, 32, 4>(), variant<P3, 1, 64, 4>()},
      {variant<D1, 1, 16, 4>(), variant<D1, 1, 32, 4>(), variant<D1, 1, 64, 2>()},
      {variant<D2, 2, 16, 5>(), variant<D2, 1, 32, 4>(), variant<D2, 2, 32, 4>(), variant<D2, 1, 64, 4>(),
       variant<D2, 1, 128, 3>()},
      {variant<D3, 2, 16, 5>(), variant<D3, 1, 32, 4>(), variant<D3, 2, 32, 4>(), variant<D3, 1, 64, 4>(),
       variant<D3, 1, 128, 3>()},
      {variant<D4, 2, 16, 5>(), variant<D4, 1, 32, 4>(), variant<D4, 2, 32, 4>(), variant<D4, 1, 64, 4>()}};
  // BF16 operands (open boundary): the same tilings; a K chunk holds 64 elements
  static const std::vector<Variant> b[4] = {
      {variant<P1, 1, 16, 4, E_BF16>(), variant<P1, 1, 32, 4, E_BF16>(), variant<P1, 1, 64, 2, E_BF16>(),
       variant<P1, 2, 16, 4, E_BF16>()},
      {variant<P2A, 2, 16, 5, E_BF16>(), variant<P2A, 1, 32, 4, E_BF16>(), variant<P2A, 2, 32, 4, E_BF16>(),
       variant<P2A, 1, 64, 4, E_BF16>(), variant<P2A, 1, 128, 3, E_BF16>()},
      {variant<P2B, 4, 16, 5, E_BF16>(), variant<P2B, 2, 32, 4, E_BF16>(), variant<P2B, 1, 64, 4, E_BF16>(),
       variant<P2B, 2, 64, 4, E_BF16>(), variant<P2B, 1, 128, 3, E_BF16>()},
      {variant<P3, 2, 16, 5, E_BF16>(), variant<P3, 1, 32, 4, E_BF16>(), variant<P3, 2, 32, 4, E_BF16>(),
       variant<P3, 1, 64, 4, E_BF16>()}};
  return (el == E_BF16 && ph <= P3) ? b[ph] : v[ph];
}

sc_status set_attrs(const Variant& v) {
  SC_CUDA(cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, v.smem));
  if (v.sk > 1) SC_CUDA(cudaFuncSetAttribute(v.fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 0));
  return SC_OK;
}

// CTAs (tiles x SK), clusters of SK along x, optionally programmatic dependent launch.
cudaError_t launch_run(int ph, const PhaseRun& r, cudaStream_t s, bool pdl) {
  const Variant& v = variants(ph, r.el)[r.variant];
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(r.grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = v.smem;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  int na = 0;
  at[na].id = cudaLaunchAttributeClusterDimension;
  at[na].val.clusterDim.x = v.sk;
  at[na].val.clusterDim.y = 1;
  at[na].val.clusterDim.z = 1;
  ++na;
  if (pdl) {
    at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  cfg.attrs = at;
  cfg.numAttrs = na;
  void* args[1] = {(void*)&r.a};
  return cudaLaunchKernelExC(&cfg, v.fn, args);
}

void host_fft(std::complex<double>* a, int n, int stride) {
  for (int i = 1, j = 0; i < n; ++i) {
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[(size_t)i * stride], a[(size_t)j * stride]);
  }
  for (int len = 2; len <= n; len <<= 1) {
    const double ang = -2.0 * M_PI / len;
    for (int i = 0; i < n; i += len)
      for (int k = 0; k < len / 2; ++k) {
        const std::complex<double> w(std::cos(ang * k), std::sin(ang * k));
        std::complex<double>& u = a[(size_t)(i + k) * stride];
        std::complex<double>& v = a[(size_t)(i + k + len / 2) * stride];
        const std::complex<double> t = v * w;
        v = u - t;
        u = u + t;
      }
  }
}

}  // namespace

// Arguments of phase ph for candidate k on grid g (tensor maps with the
// variant's tile width); SC_ERR_ARG when the variant does not fit the grid.
sc_status make_run(sc_grid* g, int ph, int k, PhaseRun& out) {
  Tf32Plan* T = g->tf32;
  const int el = T->el, kc = kc_of(el);
  const Variant& v = variants(ph, el)[k];
  const int nx = g->nx, ny = g->ny, nz = g->nstack, My = T->My, Npad = T->Npad, K3 = T->K3;
  GemmArgs& a = out.a;
  std::memset(&a, 0, sizeof a);
  a.nx = nx;
  a.ny = ny;
  a.My = My;
  a.Npad = Npad;
  a.err = T->err;
  int M = 0;
  sc_status st = SC_OK;
  switch (ph) {
    case P1:  // C[c][(s,j)] = B1 q^T: M = 2nx (c), N = nz ny (j of every stacked grid), K = nx
      if (ny % v.nt) return set_error(SC_ERR_ARG, "tile wider than a grid's rows");
      if ((st = make_map(&a.tA_hi, T->B1.hi, 2 * nx, nx, TM, el)) || (st = make_map(&a.tA_lo, T->B1.lo, 2 * nx, nx, TM, el)))
        return st;
      M = 2 * nx;
      a.k_chunks = nx / kc;
      a.n_total = nz * ny;
      a.Q = g->Q;
      a.qfac = 1.f;
      a.out_hi = T->B2.hi;
      a.out_lo = T->B2.lo;
      a.out_ld = 2 * ny;
      a.out_slice = (long long)Npad * 2 * ny;
      break;
    case P2A:  // C[r][(s,p)] = W2f B2^T: M = 2My as (Re, Im) halves, N = nz Npad, K = 2ny
      if ((st = make_map(&a.tA_hi, T->W2f.hi, 2 * My, 2 * ny, TM, el)) ||
          (st = make_map(&a.tA_lo, T->W2f.lo, 2 * My, 2 * ny, TM, el)) ||
          (st = make_map(&a.tB_hi, T->B2.hi, nz * Npad, 2 * ny, v.nt, el)) ||
          (st = make_map(&a.tB_lo, T->B2.lo, nz * Npad, 2 * ny, v.nt, el)))
        return st;
      M = 2 * My;
      a.k_chunks = 2 * ny / kc;
      a.n_total = nz * Npad;
      a.qcells = (long long)nz * nx * ny;
      a.Sx = T->Sx;
      a.Sy = T->Sy;
      a.out_hi = T->B3.hi;
      a.out_lo = T->B3.lo;
      a.out_ld = 2 * My;
      a.out_slice = (long long)2 * Npad * 2 * My;
      break;
    case P2B:  // C[r][(s,f,p)] = W2i B3^T: M = 2ny as (Re, Im) halves, N = nz 2 Npad, K = 2My
      if ((st = make_map(&a.tA_hi, T->W2i.hi, 2 * ny, 2 * My, TM, el)) ||
          (st = make_map(&a.tA_lo, T->W2i.lo, 2 * ny, 2 * My, TM, el)) ||
          (st = make_map(&a.tB_hi, T->B3.hi, nz * 2 * Npad, 2 * My, v.nt, el)) ||
          (st = make_map(&a.tB_lo, T->B3.lo, nz * 2 * Npad, 2 * My, v.nt, el)))
        return st;
      M = 2 * ny;
      a.k_chunks = 2 * My / kc;
      a.n_total = nz * 2 * Npad;
      a.out_hi = T->A3.hi;
      a.out_lo = T->A3.lo;
      a.out_ld = K3;
      a.out_slice = (long long)2 * ny * K3;
      break;
    case D1:  // T1[p][(s,j)] = S F^T: M = mp (p), N = nz mp (interior rows j of every grid), K = mp (i)
    case D2:  // W[q][(s,p)] = S T1^T, / lambda -> UT: M = mp (q), N = nz mp, K = mp (j)
    case D3:  // T3[j][(s,p)] = S UT^T: M = mp (j), N = nz mp, K = mp (q)
    case D4: {  // u[(s,j)][i] = T3 S^T: M = nz mp, N = mp (i), K = mp (p)
      const int mp = T->mp;
      if (mp % v.nt) return set_error(SC_ERR_ARG, "tile width does not divide the padded interior");
      a.m = T->m;
      a.mp = mp;
      a.k_chunks = mp / kc;
      a.out_ld = mp;
      a.out_slice = (long long)mp * mp;
      if (ph == D1 || ph == D2) {
        if ((st = make_map(&a.tA_hi, T->S.hi, mp, mp, TM, el)) || (st = make_map(&a.tA_lo, T->S.lo, mp, mp, TM, el))) return st;
        M = mp;
        a.n_total = nz * mp;
      }
      if (ph == D1) {
        a.Q = g->Q;
        a.qfac = (float)(-2.0 * M_PI / (g->hx * g->hy));
        a.out_hi = T->T1.hi;
        a.out_lo = T->T1.lo;
      } else if (ph == D2) {
        if ((st = make_map(&a.tB_hi, T->T1.hi, nz * mp, mp, v.nt, el)) || (st = make_map(&a.tB_lo, T->T1.lo, nz * mp, mp, v.nt, el)))
          return st;
        a.inv_lam = T->inv_lam;
        a.qcells = (long long)nz * nx * ny;
        a.out_hi = T->UT.hi;
        a.out_lo = T->UT.lo;
      } else if (ph == D3) {  // A = [S; Cy]: rows (f, j), the potential part and its y-derivative
        if ((st = make_map(&a.tA_hi, T->SCy.hi, 2 * mp, mp, TM, el)) || (st = make_map(&a.tA_lo, T->SCy.lo, 2 * mp, mp, TM, el)) ||
            (st = make_map(&a.tB_hi, T->UT.hi, nz * mp, mp, v.nt, el)) || (st = make_map(&a.tB_lo, T->UT.lo, nz * mp, mp, v.nt, el)))
          return st;
        M = 2 * mp;
        a.n_total = nz * mp;
        a.out_hi = T->T3.hi;
        a.out_lo = T->T3.lo;
        a.out_slice = (long long)2 * mp * mp;
      } else {  // D4: A = T3 rows (s, f, j), B = [S; Cx]: columns (h, i)
        if ((st = make_map(&a.tA_hi, T->T3.hi, nz * 2 * mp, mp, TM, el)) ||
            (st = make_map(&a.tA_lo, T->T3.lo, nz * 2 * mp, mp, TM, el)) ||
            (st = make_map(&a.tB_hi, T->SCx.hi, 2 * mp, mp, v.nt, el)) || (st = make_map(&a.tB_lo, T->SCx.lo, 2 * mp, mp, v.nt, el)))
          return st;
        M = nz * 2 * mp;
        a.n_total = 2 * mp;
        a.phi = T->phi;
        a.E = (float2*)g->E;
        a.norm = (float)(4.0 / ((double)(T->m + 1) * (double)(T->m + 1)));
        a.e_slice = (long long)nx * ny;
      }
      break;
    }
    default:  // P3: C[(s,f,j)][i] = A3 B4^T: M = nz 2ny as (Ex, Ey) halves per grid, N = nx, K = K3
      if (nx % v.nt) return set_error(SC_ERR_ARG, "tile wider than a grid's columns");
      if ((st = make_map(&a.tA_hi, T->A3.hi, nz * 2 * ny, K3, TM, el)) ||
          (st = make_map(&a.tA_lo, T->A3.lo, nz * 2 * ny, K3, TM, el)) ||
          (st = make_map(&a.tB_hi, T->B4.hi, nx, K3, v.nt, el)) || (st = make_map(&a.tB_lo, T->B4.lo, nx, K3, v.nt, el)))
        return st;
      M = nz * 2 * ny;
      a.k_chunks = K3 / kc;
      a.n_total = nx;
      a.E = (float2*)g->E;
      a.e_slice = (long long)nx * ny;
      break;
  }
  if (a.k_chunks % v.sk) return set_error(SC_ERR_ARG, "K chunks do not split evenly over the cluster");
  a.m_tiles = M / TM;
  a.n_tiles = (a.n_total + v.nt - 1) / v.nt;
  const long long grid = (long long)a.m_tiles * a.n_tiles * v.sk;
  if (grid > (1LL << 30)) return set_error(SC_ERR_ARG, "too many tiles");
  out.grid = (int)grid;
  out.variant = k;
  out.el = el;
  return set_attrs(v);
}

// Time every candidate of every phase on this grid (zero inputs; the time of a
// dense contraction does not depend on the values) and keep the fastest.
// Tiling choice, in two stages.  (1) Each phase alone: every variant that fits
// the grid, 8 back-to-back launches, best of three rounds.  (2) The whole
// solve as the turn runs it (the four phases chained by programmatic
// dependent launch): one phase at a time, each of its variants with the other
// phases' current choices, 4 chained solves per timing, best of three rounds,
// keeping the fastest (coordinate descent from the stage-1 choice).  Variants
// of a phase differ only in the FP32 summation order of split-K partial tiles,
// so the choice is made once per device and grid geometry in a process and
// every later grid of that geometry takes it: grids of one geometry give the
// same bits (near-equal timings could otherwise tip two grids different ways).
struct TuneKey {
  int dev, pipe, el, nx, ny, nstack;
  bool operator<(const TuneKey& o) const {
    return std::tie(dev, pipe, el, nx, ny, nstack) < std::tie(o.dev, o.pipe, o.el, o.nx, o.ny, o.nstack);
  }
};
struct TuneChoice {
  int variant[4];
  float us[4];
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneChoice> g_tune_choice;

sc_status tf32_tune(sc_grid* g) {
  Tf32Plan* T = g->tf32;
  int dev = 0;
  SC_CUDA(cudaGetDevice(&dev));
  const TuneKey key{dev, T->pipe ? 1 : 0, T->el, g->nx, g->ny, g->nstack};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    const auto it = g_tune_choice.find(key);
    if (it != g_tune_choice.end()) {
      for (int c = 0; c < 4; ++c) {
        PhaseRun r;
        const sc_status st = make_run(g, T->base() + c, it->second.variant[c], r);
        if (st) return st;
        T->run[c] = r;
        T->tuned_us[c] = it->second.us[c];
      }
      return SC_OK;
    }
  }
  cudaEvent_t e0, e1;
  SC_CUDA(cudaEventCreate(&e0));
  SC_CUDA(cudaEventCreate(&e1));
  sc_status st = SC_OK;
  // best of three rounds of `reps` calls of launch(), in microseconds per call
  auto timed = [&](auto&& launch, int reps, float* us) -> cudaError_t {
    cudaError_t e = launch();  // warm-up
    float best = 1e30f;
    for (int round = 0; round < 3 && e == cudaSuccess; ++round) {
      float ms = 0.f;
      e = cudaEventRecord(e0, g->stream);
      for (int i = 0; i < reps && e == cudaSuccess; ++i) e = launch();
      if (e == cudaSuccess) e = cudaEventRecord(e1, g->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      best = std::min(best, 1e3f * ms / reps);
    }
    *us = best;
    return e;
  };
  constexpr int kMaxVariants = 8;
  float iso[4][kMaxVariants] = {};  // stage-1 time of each variant
  for (int c = 0; c < 4 && !st; ++c) {
    const int ph = T->base() + c;
    float best = 1e30f;
    for (int k = 0; k < (int)variants(ph, T->el).size() && k < kMaxVariants && !st; ++k) {
      PhaseRun r;
      if (make_run(g, ph, k, r) != SC_OK) continue;  // does not fit this grid
      r.a.scale = 1.f;
      float us = 0.f;
      const cudaError_t e = timed([&] { return launch_run(ph, r, g->stream, false); }, 8, &us);
      if (e != cudaSuccess) {
        st = cuda_error(e, "tuning the split-TF32 solve");
        break;
      }
      iso[c][k] = us;
      if (us < best) {
        best = us;
        T->run[c] = r;
        T->tuned_us[c] = us;
      }
    }
    if (!st && T->run[c].variant < 0) st = set_error(SC_ERR_UNSUPPORTED, "no solve tiling fits this grid");
  }
  // stage 2: the chained solve
  auto chain = [&] {
    const sc_status s2 = tf32_solve(g, false);
    return s2 == SC_OK ? cudaSuccess : cudaErrorUnknown;
  };
  float chain_best = 0.f;
  if (!st) {
    const cudaError_t e = timed(chain, 4, &chain_best);
    if (e != cudaSuccess) st = cuda_error(e, "tuning the split-TF32 solve");
  }
  for (int c = 0; c < 4 && !st; ++c) {
    const int ph = T->base() + c;
    const PhaseRun keep = T->run[c];
    PhaseRun best_run = keep;
    for (int k = 0; k < (int)variants(ph, T->el).size() && k < kMaxVariants && !st; ++k) {
      if (k == keep.variant || iso[c][k] == 0.f) continue;  // the current choice, or does not fit
      PhaseRun r;
      if (make_run(g, ph, k, r) != SC_OK) continue;
      T->run[c] = r;
      float us = 0.f;
      const cudaError_t e = timed(chain, 4, &us);
      if (e != cudaSuccess) {
        st = cuda_error(e, "tuning the split-TF32 solve");
        break;
      }
      if (us < chain_best) {
        chain_best = us;
        best_run = r;
      }
    }
    T->run[c] = best_run;
    T->tuned_us[c] = iso[c][best_run.variant];
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!st && tf32_error(g)) st = set_error(SC_ERR_TIMEOUT, "tensor-core solve gave up on a bounded wait");
  if (!st) {
    TuneChoice ch;
    for (int c = 0; c < 4; ++c) {
      ch.variant[c] = T->run[c].variant;
      ch.us[c] = T->tuned_us[c];
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_choice.emplace(key, ch);  // a grid tuned at the same time by another thread keeps the first entry
  }
  return st;
}

// Conducting-pipe form (Sec. IV-B) as four dense GEMMs with the real sine
// matrix S[p][i] = sin(pi (p+1)(i+1) / (m+1)) of the m interior nodes
// (padded to mp = whole 128-row tiles): T1 = S F^T (rows), W = S T1^T (columns),
// U = W / lambda, [T3; T3y] = [S; Cy] U^T, and from [T3; T3y] [S; Cx]^T the
// potential (T3 S^T), Ex (T3 Cx^T) and Ey (T3y S^T), times 4/(m+1)^2.  Cx, Cy
// are the centred differences of the sine modes (cosine series), so the fields
// equal the centred differences of phi without forming them (no cancellation).
sc_status tf32_pipe_create(sc_grid* g) {
  const int nx = g->nx, ny = g->ny, nz = g->nstack;
  if (nx != ny || nx < 10 || nx > 258)
    return set_error(SC_ERR_UNSUPPORTED, "SC_SOLVE_PIPE_TF32X3 needs nx = ny in 10..258");
  sc_status st = get_encoder();
  if (st) return st;
  Tf32Plan* T = new (std::nothrow) Tf32Plan();
  if (!T) return set_error(SC_ERR_OOM, "host allocation failed");
  g->tf32 = T;
  T->pipe = true;
  const int m = nx - 2, mp = ((m + TM - 1) / TM) * TM;
  T->m = m;
  T->mp = mp;
  std::vector<double> S((size_t)mp * mp, 0.0);
  for (int p = 0; p < m; ++p)
    for (int i = 0; i < m; ++i) S[(size_t)p * mp + i] = std::sin(M_PI * (double)(p + 1) * (double)(i + 1) / (m + 1));
  // derivative matrices: the centred difference of sin(th (i+1)) is sin(th) cos(th (i+1)) / h, so
  // -d/dx of the sine series is the series with C[i][p] = -sin(th_p) cos(th_p (i+1)) / hx
  std::vector<double> SCy((size_t)2 * mp * mp, 0.0), SCx((size_t)2 * mp * mp, 0.0);
  for (int r = 0; r < m; ++r)
    for (int k = 0; k < m; ++k) {
      const double th = M_PI * (double)(k + 1) / (m + 1);
      SCy[(size_t)r * mp + k] = SCx[(size_t)r * mp + k] = S[(size_t)r * mp + k];
      SCy[(size_t)(mp + r) * mp + k] = -std::sin(th) * std::cos(th * (r + 1)) / g->hy;
      SCx[(size_t)(mp + r) * mp + k] = -std::sin(th) * std::cos(th * (r + 1)) / g->hx;
    }
  std::vector<float> il((size_t)mp * mp, 0.f);
  for (int q = 0; q < m; ++q)
    for (int p = 0; p < m; ++p) {
      const double sp = std::sin(M_PI * (p + 1) / (2.0 * (m + 1))), sq = std::sin(M_PI * (q + 1) / (2.0 * (m + 1)));
      il[(size_t)q * mp + p] = (float)(1.0 / (-4.0 * (sp * sp / (g->hx * g->hx) + sq * sq / (g->hy * g->hy))));
    }
  const int el = T->el;
  if ((st = upload(T->S, S, mp, mp, el)) || (st = upload(T->SCy, SCy, 2 * mp, mp, el)) ||
      (st = upload(T->SCx, SCx, 2 * mp, mp, el)) || (st = alloc_zero(T->T1, nz * mp, mp, el)) ||
      (st = alloc_zero(T->UT, nz * mp, mp, el)) || (st = alloc_zero(T->T3, nz * 2 * mp, mp, el)))
    return st;
  SC_CUDA(cudaMalloc(&T->inv_lam, il.size() * sizeof(float)));
  SC_CUDA(cudaMemcpy(T->inv_lam, il.data(), il.size() * sizeof(float), cudaMemcpyHostToDevice));
  SC_CUDA(cudaMalloc(&T->phi, (size_t)nz * nx * ny * sizeof(float)));
  SC_CUDA(cudaMemset(T->phi, 0, (size_t)nz * nx * ny * sizeof(float)));
  SC_CUDA(cudaMalloc(&T->err, sizeof(int)));
  SC_CUDA(cudaMemset(T->err, 0, sizeof(int)));
  return tf32_tune(g);
}

sc_status tf32_create(sc_grid* g) {
  if (g->precision == SC_SOLVE_PIPE_TF32X3) return tf32_pipe_create(g);
  const int nx = g->nx, ny = g->ny, nz = g->nstack;
  if (nx != ny || (nx != 64 && nx != 128 && nx != 256))
    return set_error(SC_ERR_UNSUPPORTED, "SC_SOLVE_TF32X3 and SC_SOLVE_BF16X3 need nx = ny in {64, 128, 256}");
  sc_status st = get_encoder();
  if (st) return st;
  Tf32Plan* T = new (std::nothrow) Tf32Plan();
  if (!T) return set_error(SC_ERR_OOM, "host allocation failed");
  g->tf32 = T;
  T->el = g->precision == SC_SOLVE_BF16X3 ? E_BF16 : E_TF32;
  const int el = T->el, kc = kc_of(el);
  // half-spectrum columns p = 0..nx, padded to a multiple of 16 (whole float4 groups per field)
  const int Mx = 2 * nx, My = 2 * ny, Npad = ((nx + 1 + 15) / 16) * 16;
  const int K3 = ((2 * Npad + 2 * kc - 1) / (2 * kc)) * (2 * kc);  // whole chunks for split-K up to 2
  T->Mx = Mx;
  T->My = My;
  T->Npad = Npad;
  T->K3 = K3;
  const double tp = 2.0 * M_PI;

  // P1: B1 [2nx][nx]
  std::vector<double> B1((size_t)2 * nx * nx);
  for (int c = 0; c < 2 * nx; ++c)
    for (int i = 0; i < nx; ++i)
      B1[(size_t)c * nx + i] = (c <= nx) ? std::cos(tp * c * i / Mx) : -std::sin(tp * (c - nx) * i / Mx);
  // P2A: W2f [2My][2ny]
  std::vector<double> W2f((size_t)2 * My * 2 * ny);
  for (int r = 0; r < 2 * My; ++r)
    for (int c = 0; c < 2 * ny; ++c) {
      const int k = r % My, j = c % ny;
      const double C = std::cos(tp * (double)k * j / My), S = std::sin(tp * (double)k * j / My);
      const bool re_row = r < My, re_col = c < ny;
      W2f[(size_t)r * 2 * ny + c] = re_row ? (re_col ? C : S) : (re_col ? -S : C);
    }
  // P2B: W2i [2ny][2My]
  std::vector<double> W2i((size_t)2 * ny * 2 * My);
  for (int r = 0; r < 2 * ny; ++r)
    for (int c = 0; c < 2 * My; ++c) {
      const int j = r % ny, k = c % My;
      const double C = std::cos(tp * (double)k * j / My), S = std::sin(tp * (double)k * j / My);
      const bool re_row = r < ny, re_col = c < My;
      W2i[(size_t)r * 2 * My + c] = re_row ? (re_col ? C : -S) : (re_col ? S : C);
    }
  // P3: B4 [nx][K3]
  std::vector<double> B4((size_t)nx * K3, 0.0);
  const double nrm = 1.0 / ((double)Mx * (double)My);
  for (int i = 0; i < nx; ++i)
    for (int p = 0; p <= nx; ++p) {
      const double w = (p == 0 || p == nx) ? 1.0 : 2.0;
      B4[(size_t)i * K3 + p] = w * std::cos(tp * (double)p * i / Mx) * nrm;
      B4[(size_t)i * K3 + Npad + p] = -w * std::sin(tp * (double)p * i / Mx) * nrm;
    }
  // spectra of the field kernels (imaginary parts), [My][Npad]
  std::vector<double> Dx((size_t)Mx * My), Dy((size_t)Mx * My);
  build_field_kernels(g, Dx.data(), Dy.data());
  std::vector<std::complex<double>> cx(Dx.begin(), Dx.end()), cy(Dy.begin(), Dy.end());
  for (int b = 0; b < My; ++b) {
    host_fft(cx.data() + (size_t)b * Mx, Mx, 1);
    host_fft(cy.data() + (size_t)b * Mx, Mx, 1);
  }
  for (int c = 0; c < Mx; ++c) {
    host_fft(cx.data() + c, My, Mx);
    host_fft(cy.data() + c, My, Mx);
  }
  // [p][k]: the P2A epilogue reads consecutive k across a warp
  std::vector<float> Sx((size_t)My * Npad, 0.f), Sy((size_t)My * Npad, 0.f);
  for (int k = 0; k < My; ++k)
    for (int p = 0; p <= nx; ++p) {
      Sx[(size_t)p * My + k] = (float)cx[(size_t)k * Mx + p].imag();
      Sy[(size_t)p * My + k] = (float)cy[(size_t)k * Mx + p].imag();
    }

  if ((st = upload(T->B1, B1, 2 * nx, nx, el)) || (st = upload(T->W2f, W2f, 2 * My, 2 * ny, el)) ||
      (st = upload(T->W2i, W2i, 2 * ny, 2 * My, el)) || (st = upload(T->B4, B4, nx, K3, el)) ||
      (st = alloc_zero(T->B2, nz * Npad, 2 * ny, el)) || (st = alloc_zero(T->B3, nz * 2 * Npad, 2 * My, el)) ||
      (st = alloc_zero(T->A3, nz * 2 * ny, K3, el)))
    return st;
  SC_CUDA(cudaMalloc(&T->Sx, Sx.size() * 4));
  SC_CUDA(cudaMalloc(&T->Sy, Sy.size() * 4));
  SC_CUDA(cudaMemcpy(T->Sx, Sx.data(), Sx.size() * 4, cudaMemcpyHostToDevice));
  SC_CUDA(cudaMemcpy(T->Sy, Sy.data(), Sy.size() * 4, cudaMemcpyHostToDevice));
  SC_CUDA(cudaMalloc(&T->err, sizeof(int)));
  SC_CUDA(cudaMemset(T->err, 0, sizeof(int)));

  if ((st = tf32_tune(g)) != SC_OK) return st;
  return SC_OK;
}

void tf32_destroy(sc_grid* g) {
  Tf32Plan* T = g->tf32;
  if (!T) return;
  free_mat(T->B1);
  free_mat(T->W2f);
  free_mat(T->W2i);
  free_mat(T->B4);
  free_mat(T->B2);
  free_mat(T->B3);
  free_mat(T->A3);
  cudaFree(T->Sx);
  cudaFree(T->Sy);
  free_mat(T->S);
  free_mat(T->SCy);
  free_mat(T->SCx);
  free_mat(T->T1);
  free_mat(T->UT);
  free_mat(T->T3);
  cudaFree(T->inv_lam);
  cudaFree(T->phi);
  cudaFree(T->err);
  delete T;
  g->tf32 = nullptr;
}

sc_status tf32_solve(sc_grid* g, bool zero_q) {
  Tf32Plan* T = g->tf32;
  if (!T) return set_error(SC_ERR_ARG, "grid has no TF32 solver");
  PhaseRun& r1 = T->run[0];
  r1.a.scale = (float)(1.0 / 1099511627776.0 / (double)(g->n_particles > 0 ? g->n_particles : 1));
  r1.a.stack_scale = (const float*)g->stack_scale;
  T->run[1].a.Qzero = zero_q ? g->Q : nullptr;  // P2A / D2: the charge has been read
  for (int c = 0; c < 4; ++c) T->run[c].a.drop_data_loads = T->drop_data_loads;
  for (int c = 0; c < 4; ++c) SC_CUDA(launch_run(T->base() + c, T->run[c], g->stream, true));
  if (T->pipe) {
    int dev = 0, sms = 0;
    SC_CUDA(cudaGetDevice(&dev));
    SC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t total = (int64_t)g->nstack * (2 * g->nx + 2 * (g->ny - 2));
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)sms * 4);
    SC_CUDA(launch_pdl(pipe_walls32, dim3(blocks), dim3(256), 0, g->stream, (const float*)T->phi, g->nx, g->ny,
                       g->nstack, (float)(1.0 / g->hx), (float)(1.0 / g->hy), (float2*)g->E));
  }
  return SC_OK;
}

int tf32_error(sc_grid* g) {
  if (!g->tf32) return 0;
  int e = 0;
  cudaMemcpy(&e, g->tf32->err, sizeof(int), cudaMemcpyDeviceToHost);
  return e;
}

double tf32_tensor_flops(const sc_grid* g) {
  // 2 M N K per GEMM (the chosen runs' logical sizes), three split products each
  const Tf32Plan* T = g->tf32;
  double f = 0.0;
  for (const PhaseRun& r : T->run)
    f += 2.0 * (double)r.a.m_tiles * TM * (double)r.a.n_total * (double)r.a.k_chunks * kc_of(r.el) * 3.0;
  return f;
}

int tf32_variant_count(int ph) { return (int)variants(ph).size(); }

sc_status tf32_test_bounded_waits(sc_grid* g, int enable) {
  if (!g->tf32) return set_error(SC_ERR_UNSUPPORTED, "the grid has no split-TF32 solve");
  g->tf32->drop_data_loads = enable ? 1 : 0;
  return SC_OK;
}

const float* tf32_potential(const sc_grid* g) { return (g->tf32 && g->tf32->pipe) ? g->tf32->phi : nullptr; }

sc_status tf32_read_potential(const sc_grid* g, double* out) {
  const Tf32Plan* T = g->tf32;
  if (!T || !T->pipe) return set_error(SC_ERR_UNSUPPORTED, "only pipe grids keep the potential");
  const size_t cells = (size_t)g->nstack * g->nx * g->ny;
  std::vector<float> v(cells);
  SC_CUDA(cudaMemcpy(v.data(), T->phi, cells * sizeof(float), cudaMemcpyDeviceToHost));
  for (size_t c = 0; c < cells; ++c) out[c] = v[c];
  return SC_OK;
}

sc_status tf32_get_tiling(const sc_grid* g, int* choice, std::string* desc) {
  const Tf32Plan* T = g->tf32;
  if (!T) return set_error(SC_ERR_UNSUPPORTED, "the grid has no split-TF32 solve");
  static const char* names[8] = {"row DFT", "column DFT", "inverse column DFT", "inverse row DFT",
                                 "row sine transform", "column sine transform / lambda", "inverse column sine transform",
                                 "inverse row sine transform"};
  for (int c = 0; c < 4; ++c) {
    const int k = T->run[c].variant, ph = T->base() + c;
    if (choice) choice[c] = k;
    if (desc) {
      const Variant& v = variants(ph, T->el)[k];
      char b[200];
      std::snprintf(b, sizeof b, "%s%s: %d columns x split-K %d, %d stages, %d CTAs (%.1f us)", c ? "; " : "",
                    names[ph], v.nt, v.sk, v.stages, T->run[c].grid, T->tuned_us[c]);
      *desc += b;
    }
  }
  return SC_OK;
}

sc_status tf32_set_tiling(sc_grid* g, const int* choice) {
  Tf32Plan* T = g->tf32;
  if (!T) return set_error(SC_ERR_UNSUPPORTED, "the grid has no split-TF32 solve");
  for (int c = 0; c < 4; ++c) {
    if (choice[c] < 0) continue;
    const int ph = T->base() + c;
    if (choice[c] >= (int)variants(ph, T->el).size()) return set_error(SC_ERR_ARG, "tiling variant index out of range");
    PhaseRun r;
    sc_status st = make_run(g, ph, choice[c], r);
    if (st) return st;
    T->run[c] = r;
    T->tuned_us[c] = 0.f;
  }
  return SC_OK;
}

}  // namespace sc
