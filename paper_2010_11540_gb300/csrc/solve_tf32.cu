// Open-boundary field solve as dense DFT GEMMs on the 5th-generation tensor
// cores (tcgen05, kind::tf32), operands staged by TMA into 128-byte-swizzled
// shared memory, accumulators in TMEM, 3-term split precision:
//   a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi,   a_hi = tf32(a), a_lo = tf32(a - a_hi),
// accumulated in FP32.
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
// Supported: nx = ny in {128, 256} (M tiles of 128 rows).
#include <cooperative_groups.h>
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "sc_internal.cuh"

namespace sc {

namespace {

constexpr int KC = 32;          // fp32 elements per K chunk (one 128-byte swizzle row)
constexpr int NT = 16;          // N columns per CTA tile
constexpr int TM = 128;         // rows per MMA / M tile
constexpr int kThreads = 128;   // 4 warps: TMA producer, MMA issuer, TMEM owner, all do the epilogue
constexpr long long kWaitCycles = 4000000000LL;  // bounded mbarrier waits (~2 s of SM clock), then error + bail out

enum Phase { P1 = 0, P2A = 1, P2B = 2, P3 = 3 };

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
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
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
// Instruction descriptor: D f32, A = B = tf32, both K-major, M = 128, N = NT.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NT >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
// hi/lo split of a value for the 3-term products
__device__ __forceinline__ void split(float x, float& hi, float& lo) {
  hi = tf32_round(x);
  lo = tf32_round(x - hi);
}

// byte offset of element (r, k), k < 32, in a K-major SW128 tile of 128-byte rows
__device__ __forceinline__ uint32_t sw128_offset(int r, int k) {
  return (uint32_t)(r * 128 + ((((k >> 2) ^ (r & 7)) << 4) | ((k & 3) << 2)));
}

struct GemmArgs {
  CUtensorMap tA_hi, tA_lo, tB_hi, tB_lo;  // tB_* unused for P1
  int k_chunks;   // K / KC
  int n_tiles;    // N tiles per M block
  int nx, ny, My, Npad;
  // P1: charge input
  const unsigned long long* Q;
  float scale;
  const float* stack_scale;  // per stacked grid (bunches of a batch), or NULL: scale
  // P2A: charge grid to clear for the next deposit (NULL: leave it)
  unsigned long long* Qzero;
  int qcells;
  // outputs / epilogue inputs
  float *out_hi, *out_lo;  // next phase's operand (P1: B2, P2A: B3, P2B: A3)
  int out_ld;              // its row length (K of the next phase)
  const float *Sx, *Sy;    // P2A: spectra [Npad][My]
  float2* E;               // P3: fields, float32 (Ex, Ey) per node
  int* err;                // set to 1 when a bounded wait ran out
  // longitudinal slices (blockIdx.y): rows per slice of the data operands and
  // elements per slice of the inputs / outputs
  int a_slice_rows, b_slice_rows;
  long long out_slice, q_slice, e_slice;
};

// Which operand is a constant DFT matrix (loadable before the grid dependency
// resolves) and which is the previous kernel's output.
template <int PH>
struct Roles {
  static constexpr bool CONST_A = (PH != P3);
  static constexpr bool TMA_B = (PH != P1);
};

template <int PH>
struct Smem {
  static constexpr int A_TILE = TM * 128;  // bytes of one 128-row x 32-element tile
  static constexpr int B_TILE = NT * 128;  // 2 KB
  static constexpr int STAGE = 2 * A_TILE + (Roles<PH>::TMA_B ? 2 * B_TILE : 0);
  static constexpr int STAGES = (PH == P1) ? 4 : 5;
  static constexpr int B_RESIDENT_MAX_CHUNKS = 8;  // P1: charge tiles for K up to 256
  static constexpr int RESIDENT = (PH == P1) ? 2 * B_RESIDENT_MAX_CHUNKS * B_TILE : 0;
  static constexpr int BYTES = STAGES * STAGE + RESIDENT + 1024 /*align slack*/;
};

namespace cg = cooperative_groups;
__device__ __forceinline__ void prefetch_map(const CUtensorMap* m) {
  asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)m) : "memory");
}

// One cluster of SK CTAs: a 128-row x NT-column tile of C = A B^T, the K
// chunks split evenly across the SK CTAs; each accumulates its three split
// products in TMEM, the partial tiles are summed through distributed shared
// memory and each CTA finishes NT/SK of the columns.
template <int PH, int SK>
__global__ void __launch_bounds__(kThreads, 1) dft_gemm(const __grid_constant__ GemmArgs g) {
  using L = Smem<PH>;
  using R = Roles<PH>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[L::STAGES], empty_bar[L::STAGES], accum_bar;
  __shared__ uint32_t tmem_base_s;
  __shared__ volatile int abort_s;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rank = (SK > 1) ? (int)cg::this_cluster().block_rank() : 0;
  const int tile = blockIdx.x / SK;
  const int mb = tile / g.n_tiles, nb = tile % g.n_tiles;
  const int n0 = nb * NT, a_row = mb * TM;
  const int slice = blockIdx.y;
  const int a_row_g = a_row + slice * g.a_slice_rows;  // row of the (stacked) A tensor
  const int n0_g = n0 + slice * g.b_slice_rows;        // row of the (stacked) B tensor
  unsigned char* stage_base = smem;
  unsigned char* resident = smem + L::STAGES * L::STAGE;
  const int kpc = g.k_chunks / SK, kc0 = rank * kpc;  // this CTA's K chunks: kc0 .. kc0+kpc-1
  const int pre = kpc < L::STAGES ? kpc : L::STAGES;

  auto load_a = [&](int lk, int st) {
    unsigned char* sb = stage_base + st * L::STAGE;
    tma_load_2d(sb, &g.tA_hi, &full_bar[st], (kc0 + lk) * KC, a_row_g);
    tma_load_2d(sb + L::A_TILE, &g.tA_lo, &full_bar[st], (kc0 + lk) * KC, a_row_g);
  };
  auto load_b = [&](int lk, int st) {
    unsigned char* bb = stage_base + st * L::STAGE + 2 * L::A_TILE;
    tma_load_2d(bb, &g.tB_hi, &full_bar[st], (kc0 + lk) * KC, n0_g);
    tma_load_2d(bb + L::B_TILE, &g.tB_lo, &full_bar[st], (kc0 + lk) * KC, n0_g);
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
  if (warp == 2) tmem_alloc(&tmem_base_s, 32);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;

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
  if (PH == P2A && g.Qzero) {
    // every reader of the charge (the row transform) has finished: clear it for the next deposit
    for (long long c = ((long long)blockIdx.y * gridDim.x + blockIdx.x) * kThreads + threadIdx.x; c < g.qcells;
         c += (long long)gridDim.x * gridDim.y * kThreads)
      g.Qzero[c] = 0ull;
  }
  if (PH == P1) {
    // B operand = normalised charge rows j = n0 .. n0+NT-1, all K = nx, split hi/lo, swizzled.
    // 16-byte loads, all issued before any is used.
    constexpr int PER2 = NT * 256 / 2 / kThreads;  // pairs per thread for nx <= 256
    const int pairs = NT * g.nx / 2;
    const longlong2* q2 = (const longlong2*)(g.Q + slice * g.q_slice + (size_t)n0 * g.nx);
    const float qscale = g.stack_scale ? g.stack_scale[slice] : g.scale;
    longlong2 v[PER2];
#pragma unroll
    for (int u = 0; u < PER2; ++u) {
      const int e = threadIdx.x + u * kThreads;
      v[u] = (e < pairs) ? q2[e] : make_longlong2(0, 0);
    }
#pragma unroll
    for (int u = 0; u < PER2; ++u) {
      const int e = threadIdx.x + u * kThreads;
      if (e < pairs) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const unsigned long long qi = (unsigned long long)(h ? v[u].y : v[u].x);
          const int el = 2 * e + h, r = el / g.nx, i = el % g.nx;
          // uint64 -> float through its 32-bit halves (no FP64 instruction)
          const float qv =
              fmaf(__uint2float_rn((unsigned)(qi >> 32)), 4294967296.f, __uint2float_rn((unsigned)qi)) * qscale;
          float hi, lo;
          split(qv, hi, lo);
          const int kc = i / KC, k = i % KC;
          *(float*)(resident + (2 * kc) * L::B_TILE + sw128_offset(r, k)) = hi;
          *(float*)(resident + (2 * kc + 1) * L::B_TILE + sw128_offset(r, k)) = lo;
        }
      }
    }
    fence_proxy_async();
  }
  __syncthreads();

  if (warp == 0 && lane == 0) {
    // ---- TMA producer: the data operand of the prefetched stages, then whole stages
    for (int kc = 0; kc < pre; ++kc) {
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
      const unsigned char* bh = (PH == P1) ? resident + (2 * (kc0 + kc)) * L::B_TILE : sb + 2 * L::A_TILE;
      const unsigned char* bl = bh + L::B_TILE;
      const uint64_t dbh = desc_sw128(smem_u32(bh)), dbl = desc_sw128(smem_u32(bl));
      const uint64_t dah = desc_sw128(smem_u32(sb)), dal = desc_sw128(smem_u32(sb + L::A_TILE));
#pragma unroll
      for (int kk = 0; kk < KC / 8; ++kk) {
        const uint64_t o = (uint64_t)(kk * 2);  // 32 bytes per K step, in 16-byte units
        mma_tf32(tmem, dah + o, dbh + o, kIdesc, (kc > 0 || kk > 0) ? 1u : 0u);
        mma_tf32(tmem, dah + o, dbl + o, kIdesc, 1u);
        mma_tf32(tmem, dal + o, dbh + o, kIdesc, 1u);
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
  const bool have = mbar_wait(&accum_bar, 0);
  if ((!have || abort_s) && threadIdx.x == 0) atomicExch(g.err, 1);
  tc_fence_after();
  const int t = warp * 32 + lane;
  const int r = a_row + t;  // row of C
  float acc[NT];
  if (have) tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16), acc);
  constexpr int CW = NT / SK;  // columns finished by this CTA
  const int c0 = rank * CW;
  if (SK > 1) {
    // partial tiles -> shared memory (the stages are idle now), summed across the cluster
    cg::cluster_group cl = cg::this_cluster();
    float4* red = (float4*)stage_base;
#pragma unroll
    for (int q4 = 0; q4 < NT / 4; ++q4)
      red[t * (NT / 4) + q4] = have ? make_float4(acc[4 * q4], acc[4 * q4 + 1], acc[4 * q4 + 2], acc[4 * q4 + 3])
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
    cl.sync();
    float4 part[SK][CW / 4];
#pragma unroll
    for (int q = 0; q < SK; ++q) {
      const float4* rem = cl.map_shared_rank(red, q);
#pragma unroll
      for (int q4 = 0; q4 < CW / 4; ++q4) part[q][q4] = rem[t * (NT / 4) + c0 / 4 + q4];
    }
#pragma unroll
    for (int q4 = 0; q4 < CW / 4; ++q4) {
      float4 v = part[0][q4];
#pragma unroll
      for (int q = 1; q < SK; ++q) {
        v.x += part[q][q4].x;
        v.y += part[q][q4].y;
        v.z += part[q][q4].z;
        v.w += part[q][q4].w;
      }
      acc[c0 + 4 * q4] = v.x;
      acc[c0 + 4 * q4 + 1] = v.y;
      acc[c0 + 4 * q4 + 2] = v.z;
      acc[c0 + 4 * q4 + 3] = v.w;
    }
  }
  if (have && !abort_s) {
    if (PH == P1) {
      // row c of R1T: Re F1(j, p = c) for c <= nx, Im F1(j, p = c - nx) above
      const int p = (r <= g.nx) ? r : r - g.nx;
      const int half = (r <= g.nx) ? 0 : 1;
      const size_t ob = slice * g.out_slice + (size_t)p * g.out_ld + half * g.ny + n0 + c0;
      float4* dh = (float4*)(g.out_hi + ob);
      float4* dl = (float4*)(g.out_lo + ob);
#pragma unroll
      for (int q4 = 0; q4 < CW / 4; ++q4) {
        float h[4], l[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) split(acc[c0 + 4 * q4 + u], h[u], l[u]);
        dh[q4] = make_float4(h[0], h[1], h[2], h[3]);
        dl[q4] = make_float4(l[0], l[1], l[2], l[3]);
      }
    } else if (PH == P2A) {
      // row r < My: Re F(k = r, p) -> Im H_f = S_f Re F (column My + k of B3)
      // row r >= My: Im F(k = r - My, p) -> Re H_f = -S_f Im F (column k)
      const bool re = r < g.My;
      const int k = re ? r : r - g.My;
      const int col = re ? g.My + k : k;
      const float sgn = re ? 1.f : -1.f;
      // all spectrum loads first (the stores below could alias them for the compiler)
      float sx[CW], sy[CW];
#pragma unroll
      for (int cc = 0; cc < CW; ++cc) {
        sx[cc] = __ldg(g.Sx + (size_t)(n0 + c0 + cc) * g.My + k);
        sy[cc] = __ldg(g.Sy + (size_t)(n0 + c0 + cc) * g.My + k);
      }
#pragma unroll
      for (int cc = 0; cc < CW; ++cc) {
        const int p = n0 + c0 + cc;
        const float f = sgn * acc[c0 + cc];
        const size_t rx = slice * g.out_slice + (size_t)p * g.out_ld + col;
        const size_t ry = slice * g.out_slice + (size_t)(g.Npad + p) * g.out_ld + col;
        split(sx[cc] * f, g.out_hi[rx], g.out_lo[rx]);
        split(sy[cc] * f, g.out_hi[ry], g.out_lo[ry]);
      }
    } else if (PH == P2B) {
      // row r: part (Re G, Im G) = r / ny at j' = r % ny; columns n = f*Npad + p
      const int part = r / g.ny, jr = r % g.ny;
      const int f = n0 / g.Npad, p0 = n0 % g.Npad;  // NT divides Npad: one field per tile
      const size_t o = slice * g.out_slice + (size_t)(f * g.ny + jr) * g.out_ld + part * g.Npad + p0 + c0;
      float4* dh = (float4*)(g.out_hi + o);
      float4* dl = (float4*)(g.out_lo + o);
#pragma unroll
      for (int q4 = 0; q4 < CW / 4; ++q4) {
        float h[4], l[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) split(acc[c0 + 4 * q4 + u], h[u], l[u]);
        dh[q4] = make_float4(h[0], h[1], h[2], h[3]);
        dl[q4] = make_float4(l[0], l[1], l[2], l[3]);
      }
    } else {
      // row r: field f = r / ny (Ex, Ey) at j = r % ny; columns i = n0 + cc; float32 (Ex, Ey) pairs
      const int f = r / g.ny, j = r % g.ny;
      float* e = (float*)g.E + 2 * (slice * g.e_slice + (size_t)j * g.nx + n0) + f;
#pragma unroll
      for (int cc = c0; cc < c0 + CW; ++cc) e[2 * cc] = acc[cc];
    }
  }
  if (SK > 1) cg::this_cluster().sync();  // keep this CTA's partial tile alive until every rank has read it
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tmem, 32);
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

// 2-D fp32 row-major [rows][cols] tensor map with boxes of 32 x box_rows, 128-byte swizzle.
sc_status make_map(CUtensorMap* tm, const float* base, int rows, int cols, int box_rows) {
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * sizeof(float)};
  cuuint32_t box[2] = {(cuuint32_t)KC, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, es,
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

void split_host(const std::vector<double>& a, std::vector<float>& hi, std::vector<float>& lo) {
  hi.resize(a.size());
  lo.resize(a.size());
  for (size_t i = 0; i < a.size(); ++i) {
    hi[i] = tf32_host((float)a[i]);
    lo[i] = tf32_host((float)(a[i] - (double)hi[i]));
  }
}

struct Mat {
  float* hi = nullptr;
  float* lo = nullptr;
  int rows = 0, cols = 0;
};

}  // namespace

struct Tf32Plan {
  int Mx, My, Npad;
  Mat B1, W2f, W2i, B4;      // constants
  Mat B2, B3, A3;            // intermediates (next phase operands)
  float *Sx, *Sy;            // [Npad][My]
  int K3;                    // row length of A3 and B4 (2 Npad rounded up to whole split-K chunks)
  int* err;
  GemmArgs a1, a2a, a2b, a3;
  int grid1, grid2a, grid2b, grid3;
};

namespace {

sc_status upload(Mat& m, const std::vector<double>& v, int rows, int cols) {
  std::vector<float> hi, lo;
  split_host(v, hi, lo);
  m.rows = rows;
  m.cols = cols;
  SC_CUDA(cudaMalloc(&m.hi, hi.size() * 4));
  SC_CUDA(cudaMalloc(&m.lo, lo.size() * 4));
  SC_CUDA(cudaMemcpy(m.hi, hi.data(), hi.size() * 4, cudaMemcpyHostToDevice));
  SC_CUDA(cudaMemcpy(m.lo, lo.data(), lo.size() * 4, cudaMemcpyHostToDevice));
  return SC_OK;
}

sc_status alloc_zero(Mat& m, int rows, int cols) {
  m.rows = rows;
  m.cols = cols;
  SC_CUDA(cudaMalloc(&m.hi, (size_t)rows * cols * 4));
  SC_CUDA(cudaMalloc(&m.lo, (size_t)rows * cols * 4));
  SC_CUDA(cudaMemset(m.hi, 0, (size_t)rows * cols * 4));
  SC_CUDA(cudaMemset(m.lo, 0, (size_t)rows * cols * 4));
  return SC_OK;
}

void free_mat(Mat& m) {
  cudaFree(m.hi);
  cudaFree(m.lo);
  m = Mat{};
}

// Split-K cluster size per phase (K chunks per CTA: P1 nx/32, P2A 2ny/64, P2B 2My/128, P3 K3/64).
constexpr int SK1 = 1, SK2A = 2, SK2B = 4, SK3 = 2;

template <int PH, int SK>
sc_status set_smem_attr() {
  SC_CUDA(cudaFuncSetAttribute(dft_gemm<PH, SK>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<PH>::BYTES));
  if (SK > 1) SC_CUDA(cudaFuncSetAttribute(dft_gemm<PH, SK>, cudaFuncAttributeNonPortableClusterSizeAllowed, 0));
  return SC_OK;
}

// tiles x SK CTAs, clusters of SK along x, programmatic dependent launch.
template <int PH, int SK>
cudaError_t launch_phase(int tiles, int slices, const GemmArgs& a, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(tiles * SK, slices);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = Smem<PH>::BYTES;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  at[1].id = cudaLaunchAttributeClusterDimension;
  at[1].val.clusterDim.x = SK;
  at[1].val.clusterDim.y = 1;
  at[1].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, dft_gemm<PH, SK>, a);
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

sc_status tf32_create(sc_grid* g) {
  const int nx = g->nx, ny = g->ny, nz = g->nstack;
  if (nx != ny || (nx != 64 && nx != 128 && nx != 256))
    return set_error(SC_ERR_UNSUPPORTED, "SC_SOLVE_TF32X3 needs nx = ny in {64, 128, 256}");
  sc_status st = get_encoder();
  if (st) return st;
  Tf32Plan* T = new (std::nothrow) Tf32Plan();
  if (!T) return set_error(SC_ERR_OOM, "host allocation failed");
  g->tf32 = T;
  const int Mx = 2 * nx, My = 2 * ny, Npad = ((nx + 1 + NT - 1) / NT) * NT;
  const int K3 = ((2 * Npad + KC * SK3 - 1) / (KC * SK3)) * (KC * SK3);
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

  if ((st = upload(T->B1, B1, 2 * nx, nx)) || (st = upload(T->W2f, W2f, 2 * My, 2 * ny)) ||
      (st = upload(T->W2i, W2i, 2 * ny, 2 * My)) || (st = upload(T->B4, B4, nx, K3)) ||
      (st = alloc_zero(T->B2, nz * Npad, 2 * ny)) || (st = alloc_zero(T->B3, nz * 2 * Npad, 2 * My)) ||
      (st = alloc_zero(T->A3, nz * 2 * ny, K3)))
    return st;
  SC_CUDA(cudaMalloc(&T->Sx, Sx.size() * 4));
  SC_CUDA(cudaMalloc(&T->Sy, Sy.size() * 4));
  SC_CUDA(cudaMemcpy(T->Sx, Sx.data(), Sx.size() * 4, cudaMemcpyHostToDevice));
  SC_CUDA(cudaMemcpy(T->Sy, Sy.data(), Sy.size() * 4, cudaMemcpyHostToDevice));
  SC_CUDA(cudaMalloc(&T->err, sizeof(int)));
  SC_CUDA(cudaMemset(T->err, 0, sizeof(int)));

  auto base = [&](GemmArgs& a) {
    std::memset(&a, 0, sizeof a);
    a.nx = nx;
    a.ny = ny;
    a.My = My;
    a.Npad = Npad;
    a.err = T->err;
    a.q_slice = (long long)nx * ny;
    a.e_slice = (long long)nx * ny;
  };
  // P1: C[c][j] = B1 q^T: M = 2nx (c), N = ny (j), K = nx
  base(T->a1);
  if ((st = make_map(&T->a1.tA_hi, T->B1.hi, 2 * nx, nx, TM)) || (st = make_map(&T->a1.tA_lo, T->B1.lo, 2 * nx, nx, TM)))
    return st;
  T->a1.k_chunks = nx / KC;
  T->a1.n_tiles = ny / NT;
  T->a1.Q = g->Q;
  T->a1.out_hi = T->B2.hi;
  T->a1.out_lo = T->B2.lo;
  T->a1.out_ld = 2 * ny;
  T->a1.out_slice = (long long)Npad * 2 * ny;
  T->grid1 = (2 * nx / TM) * T->a1.n_tiles;
  // P2A: C[r][p] = W2f B2^T: M = 2My as (Re, Im) pairs of 128 rows, N = Npad, K = 2ny
  base(T->a2a);
  if ((st = make_map(&T->a2a.tA_hi, T->W2f.hi, 2 * My, 2 * ny, TM)) ||
      (st = make_map(&T->a2a.tA_lo, T->W2f.lo, 2 * My, 2 * ny, TM)) ||
      (st = make_map(&T->a2a.tB_hi, T->B2.hi, nz * Npad, 2 * ny, NT)) ||
      (st = make_map(&T->a2a.tB_lo, T->B2.lo, nz * Npad, 2 * ny, NT)))
    return st;
  T->a2a.k_chunks = 2 * ny / KC;
  T->a2a.n_tiles = Npad / NT;
  T->a2a.Qzero = nullptr;
  T->a2a.qcells = nz * nx * ny;
  T->a2a.Sx = T->Sx;
  T->a2a.Sy = T->Sy;
  T->a2a.out_hi = T->B3.hi;
  T->a2a.out_lo = T->B3.lo;
  T->a2a.out_ld = 2 * My;
  T->a2a.b_slice_rows = Npad;
  T->a2a.out_slice = (long long)2 * Npad * 2 * My;
  T->grid2a = (2 * My / TM) * T->a2a.n_tiles;
  // P2B: C[r][(f,p)] = W2i B3^T: M = 2ny as (Re, Im) pairs, N = 2 Npad, K = 2My
  base(T->a2b);
  if ((st = make_map(&T->a2b.tA_hi, T->W2i.hi, 2 * ny, 2 * My, TM)) ||
      (st = make_map(&T->a2b.tA_lo, T->W2i.lo, 2 * ny, 2 * My, TM)) ||
      (st = make_map(&T->a2b.tB_hi, T->B3.hi, nz * 2 * Npad, 2 * My, NT)) ||
      (st = make_map(&T->a2b.tB_lo, T->B3.lo, nz * 2 * Npad, 2 * My, NT)))
    return st;
  T->a2b.k_chunks = 2 * My / KC;
  T->a2b.n_tiles = 2 * Npad / NT;
  T->a2b.out_hi = T->A3.hi;
  T->a2b.out_lo = T->A3.lo;
  T->a2b.out_ld = K3;
  T->a2b.b_slice_rows = 2 * Npad;
  T->a2b.out_slice = (long long)2 * ny * K3;
  T->grid2b = (2 * ny / TM) * T->a2b.n_tiles;
  // P3: C[(f,j)][i] = A3 B4^T: M = 2ny as (Ex, Ey) pairs, N = nx, K = 2 Npad
  base(T->a3);
  if ((st = make_map(&T->a3.tA_hi, T->A3.hi, nz * 2 * ny, K3, TM)) ||
      (st = make_map(&T->a3.tA_lo, T->A3.lo, nz * 2 * ny, K3, TM)) ||
      (st = make_map(&T->a3.tB_hi, T->B4.hi, nx, K3, NT)) || (st = make_map(&T->a3.tB_lo, T->B4.lo, nx, K3, NT)))
    return st;
  T->a3.k_chunks = K3 / KC;
  T->a3.a_slice_rows = 2 * ny;
  T->a3.n_tiles = nx / NT;
  T->a3.E = (float2*)g->E;
  T->grid3 = (2 * ny / TM) * T->a3.n_tiles;
  if ((st = set_smem_attr<P1, SK1>()) || (st = set_smem_attr<P2A, SK2A>()) || (st = set_smem_attr<P2B, SK2B>()) ||
      (st = set_smem_attr<P3, SK3>()))
    return st;
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
  cudaFree(T->err);
  delete T;
  g->tf32 = nullptr;
}

sc_status tf32_solve(sc_grid* g, bool zero_q) {
  Tf32Plan* T = g->tf32;
  if (!T) return set_error(SC_ERR_ARG, "grid has no TF32 solver");
  T->a1.scale = (float)(1.0 / 1099511627776.0 / (double)(g->n_particles > 0 ? g->n_particles : 1));
  T->a1.stack_scale = (const float*)g->stack_scale;
  T->a2a.Qzero = zero_q ? g->Q : nullptr;
  SC_CUDA((launch_phase<P1, SK1>(T->grid1, g->nstack, T->a1, g->stream)));
  SC_CUDA((launch_phase<P2A, SK2A>(T->grid2a, g->nstack, T->a2a, g->stream)));
  SC_CUDA((launch_phase<P2B, SK2B>(T->grid2b, g->nstack, T->a2b, g->stream)));
  SC_CUDA((launch_phase<P3, SK3>(T->grid3, g->nstack, T->a3, g->stream)));
  return SC_OK;
}

int tf32_error(sc_grid* g) {
  if (!g->tf32) return 0;
  int e = 0;
  cudaMemcpy(&e, g->tf32->err, sizeof(int), cudaMemcpyDeviceToHost);
  return e;
}

}  // namespace sc
