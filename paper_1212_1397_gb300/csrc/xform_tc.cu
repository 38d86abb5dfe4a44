// x/y eigen-transforms of the preconditioner (Eq. 3DAP) on the 5th-generation tensor cores.
//
// One transform contracts every row of a planar FP32 field along its contiguous axis with
// the real basis matrix B (P modes x K points):  out(row, p) = sum_k in(row, k) B(p, k).
// It is a GEMM  D[M x N] = A[M x K] B[N x K]^T  with A = data rows (K-major) and B = basis
// (K-major).  Split precision: each FP32 value x is written to shared memory as BF16
// hi = bf16(x) and lo = bf16(x - hi); the basis is split the same way on the host, and
// D accumulates hi*hi + lo*hi (+ hi*lo) in FP32 in tensor memory (1, 2 or 3 products).
//
// Persistent and warp-specialised: one CTA per SM walks the work items (128-row tile x
// column group) blockIdx.x, + gridDim.x, ...; K is streamed in 32-element stages through
// three rings in shared memory:
//   * eight converter warps (warp w <-> rows 16 w .. 16 w + 15 of the tile) copy their rows'
//     32 FP32 values of a stage into an FP32 ring with cp.async, three stages ahead (each
//     instruction of a warp covers whole 128-byte row segments), then split them (half a
//     row per thread) into the BF16 hi/lo operand ring (no-swizzle K-major core matrices:
//     8 rows x 16 bytes, 8-row groups 128 B apart, K step one column of core matrices) and
//     arrive on the stage's `afull` mbarrier.  Output columns beyond 256 (at most 8, the
//     258-point Neumann axes) are accumulated in FP32 by the same threads from the values
//     they already hold, and written by them;
//   * one producer thread streams the basis stage (hi and lo tiles, prepared on the host)
//     into the basis ring with cp.async.bulk completing on `bfull`;
//   * one MMA thread waits for both, issues the tcgen05.mma's of the stage into one of two
//     256-column tensor-memory accumulators and commits them to `sfree` (which releases the
//     stage's operand slots) and, after a tile's last stage, to `tfull`;
//   * eight epilogue warps drain the other accumulator (tcgen05.ld, 32 lanes = 32 rows per
//     warp, two warps per lane quarter taking alternate 16-column chunks) while the next
//     tile's MMAs run, store it either transposed within planes of R rows
//     (out[(row/R)*R*P + p*R + row%R]: consecutive lanes on consecutive addresses) or
//     row-major through a per-warp shared-memory transpose (out[row*P + p]: row segments
//     written by consecutive lanes), and release it on `tempty`.  The global stores are
//     the slowest part of a tile (measured), hence eight warps issuing them.
// Every mbarrier wait is bounded and warp-uniform; a timeout sets a shared flag that ends
// every role's loop, and *err for the host.  Whatever the path, the MMA thread waits
// (bounded) for all of its committed MMAs, the producer for its last bulk copy and the
// converters for their cp.async groups before the tensor memory is freed.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "helm6_internal.h"

namespace helm6 {

namespace {

constexpr int TC_M = 128;
constexpr int TC_KT = 32;                // K per stage
constexpr int TC_KC = TC_KT / 8;         // core-matrix columns per stage
constexpr int TC_GMAX = 256;             // output columns of one work item (MMA N limit)
constexpr int TC_TAILMAX = 8;            // FP32 columns beyond 256 done by the converters
constexpr int NS = 3;                    // operand ring stages (data hi/lo and basis)
constexpr int ND = 3;                    // FP32 data ring stages (cp.async in flight)
constexpr int EPI_WARPS = 8;             // warps 0-7: epilogue (lane quarter w % 4, column half w / 4)
constexpr int CONV_WARPS = 8;            // warps 8-15: converters (16 tile rows each)
constexpr int W_PROD = 16, W_MMA = 17;   // basis producer, MMA issuer + TMEM owner
constexpr int TC_THREADS = 576;
constexpr int A_TILE = TC_M * TC_KT * 2;            // bytes of one BF16 term of a data stage
constexpr int A_STAGE = 2 * A_TILE;                 // hi + lo
constexpr int A_LBO = (TC_M / 8) * 128;             // K step of the data stage
constexpr int B_STAGE = 2 * TC_KC * TC_GMAX * 16;   // hi + lo basis, 256 rows
constexpr int D_STAGE = TC_M * TC_KT * 4;           // FP32 data, 128 B per row
constexpr int EPI_COLS = 16;                        // columns per epilogue chunk
constexpr int STG_TLD = 36;                         // staged column stride of the transposed store
constexpr int STG_FLOATS = EPI_COLS * STG_TLD;      // per-warp staging (>= 32 rows x 16 columns)
constexpr int OFF_A = 0;
constexpr int OFF_B = OFF_A + NS * A_STAGE;
constexpr int OFF_D = OFF_B + NS * B_STAGE;
constexpr int OFF_T = OFF_D + ND * D_STAGE;
constexpr int TAIL_LD = ((TC_GMAX + TC_TAILMAX + TC_KT - 1) / TC_KT) * TC_KT;  // tail row stride (288)
constexpr int TAIL_FLOATS = TC_TAILMAX * TAIL_LD;
constexpr int OFF_S = OFF_T + TAIL_FLOATS * 4;
constexpr int OFF_BAR = OFF_S + EPI_WARPS * STG_FLOATS * 4;
constexpr int NBAR = 3 * NS + 5;  // afull, bfull, sfree per stage; tfull, tempty per buffer; drain
constexpr int OFF_MISC = OFF_BAR + NBAR * 8;
constexpr int SMEM_BYTES = OFF_MISC + 16 + 1024;  // + alignment of the base to 1024
static_assert(SMEM_BYTES <= 232448, "shared memory per CTA");
static_assert(OFF_B % 1024 == 0 && OFF_D % 16 == 0 && OFF_T % 16 == 0 && OFF_BAR % 8 == 0, "alignment");
constexpr int kMaxPolls = 1 << 22;

struct TcArgs {
  const float* in;
  float* out;
  const uint8_t* W;   // per column group: [kt][term][kc][Npad_g / 8][8 rows][16 B]
  const float* Bt;    // tail basis rows (FP32, tail x K) or null
  int M_total, K, P, nk, terms, transposed, R;
  int ldin;  // input row pitch (floats, >= K)
  int ldo;   // output pitch: of a row (row-major, >= P) or of a plane row of R (transposed, >= R)
  int ngroups, gcols, tail, nwork;
  int vec;  // floats per store of the epilogue: 4, 2 or 1 (from the output pitch and alignment)
  int* err;
};

__device__ __forceinline__ uint32_t s_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle: start, K step (lbo), 8-row step (sbo).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M = 128, N.
__device__ __forceinline__ uint32_t idesc(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

__device__ __forceinline__ bool try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred P1;\n mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n"
      " selp.b32 %0, 1, 0, P1;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait by one thread; gives up when the flag is raised by another role.
__device__ __forceinline__ bool poll1(uint32_t bar, uint32_t parity, volatile int* fail) {
  for (int it = 0; it < kMaxPolls; ++it) {
    if (try_wait(bar, parity)) return true;
    if ((it & 255) == 255 && *fail) return false;
  }
  *fail = 1;
  return false;
}

// Warp-uniform bounded wait: lane 0 polls, the warp takes its answer.
__device__ __forceinline__ bool pollw(uint32_t bar, uint32_t parity, volatile int* fail, int lane) {
  int ok = 0;
  if (lane == 0) ok = poll1(bar, parity, fail) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 16 consecutive tensor-memory columns of the warp's 32 lanes (one row per thread).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

template <int VEC>
__device__ __forceinline__ void cp_async(uint32_t dst, const void* src, int bytes) {
  if constexpr (VEC == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(dst), "l"(src), "n"(VEC), "r"(bytes)
                 : "memory");
}

__host__ __device__ __forceinline__ int round16(int n) { return ((n + 15) / 16) * 16; }

// Work item w of the launch: row tile w / ngroups, column group w % ngroups.
struct Item {
  int m0, grp, c0, pc, npad;
};
__device__ __forceinline__ Item item(const TcArgs& p, int w) {
  Item it;
  it.grp = w % p.ngroups;
  it.m0 = (w / p.ngroups) * TC_M;
  it.c0 = it.grp * p.gcols;
  it.pc = min(p.gcols, p.P - it.c0);
  it.npad = round16(it.pc);
  return it;
}

// Split 8 FP32 values into 8 BF16 hi (16 bytes) and 8 BF16 lo.
__device__ __forceinline__ void split8(const float4& a, const float4& b, uint4& hi, uint4& lo) {
  const float x[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
  uint32_t h[4], l[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    __nv_bfloat162 hh = __floats2bfloat162_rn(x[2 * q], x[2 * q + 1]);
    const float2 hf = __bfloat1622float2(hh);
    __nv_bfloat162 ll = __floats2bfloat162_rn(x[2 * q] - hf.x, x[2 * q + 1] - hf.y);
    h[q] = *reinterpret_cast<uint32_t*>(&hh);
    l[q] = *reinterpret_cast<uint32_t*>(&ll);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// TAIL: whether the kernel forms FP32 tail columns at all (a compile-time switch: the tail code
// left in the converter loop of a transform without tail columns costs it 10-15 %, measured;
// with tail columns the runtime test on p.tail stays, which measured faster than without)
template <int VEC, bool TAIL>
__global__ void __launch_bounds__(TC_THREADS, 1) xform_tc_kernel(TcArgs p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint64_t* bars = (uint64_t*)(smem + OFF_BAR);
  uint32_t* tslot = (uint32_t*)(smem + OFF_MISC);
  volatile int* fail = (volatile int*)(tslot + 1);
  const uint32_t bar0 = s_addr(bars);
  auto afull = [&](int s) { return bar0 + 8u * s; };             // converters stored the data stage
  auto bfull = [&](int s) { return bar0 + 8u * (NS + s); };      // basis stage arrived
  auto sfree = [&](int s) { return bar0 + 8u * (2 * NS + s); };  // the stage's MMAs completed
  auto tfull = [&](int b) { return bar0 + 8u * (3 * NS + b); };  // accumulator b complete
  auto tempty = [&](int b) { return bar0 + 8u * (3 * NS + 2 + b); };  // accumulator b drained
  const uint32_t drain = bar0 + 8u * (3 * NS + 4);                 // every MMA issued completed

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(afull(s)), "r"(CONV_WARPS));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bfull(s)), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sfree(s)), "r"(1));
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tfull(b)), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tempty(b)), "r"(EPI_WARPS));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(drain), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
    asm volatile("fence.proxy.async.shared::cta;");
    *fail = 0;
  }
  // tail basis rows, zero beyond K up to the last stage's end (K stages of 32)
  float* sBt = (float*)(smem + OFF_T);
  for (int i = tid; i < p.tail * TAIL_LD; i += TC_THREADS) {
    const int c = i / TAIL_LD, k = i - c * TAIL_LD;
    sBt[i] = k < p.K ? p.Bt[c * p.K + k] : 0.f;
  }
  if (warp == W_MMA) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(tslot)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  const int nitems = (int)blockIdx.x < p.nwork ? (p.nwork - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int nstages = nitems * p.nk;

  if (warp == W_PROD) {
    // ---- basis producer ----
    int last = -1;
    if (lane == 0) {
      int g = 0;
      for (int i = 0; i < nitems && !*fail; ++i) {
        const Item it = item(p, (int)blockIdx.x + i * (int)gridDim.x);
        const int gpad = round16(p.gcols);
        const int bterm = TC_KC * it.npad * 16;
        const int btx = (p.terms == 3 ? 2 : 1) * bterm;
        const uint8_t* Wg = p.W + (size_t)it.grp * p.nk * 2 * TC_KC * gpad * 16;
        for (int kt = 0; kt < p.nk; ++kt, ++g) {
          const int s = g % NS, u = g / NS;
          if (u >= 1 && !poll1(sfree(s), (u - 1) & 1, fail)) break;
          const uint32_t dst = s_addr(smem + OFF_B + s * B_STAGE);
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bfull(s)), "r"(btx) : "memory");
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
              "l"(Wg + (size_t)kt * 2 * bterm), "r"(btx), "r"(bfull(s))
              : "memory");
          last = g;
        }
        if (*fail) break;
      }
      // the last copy must have landed before the CTA ends
      if (last >= 0) poll1(bfull(last % NS), (last / NS) & 1, fail);
    }
    __syncwarp();
  } else if (warp == W_MMA) {
    // ---- MMA issuer ----
    if (lane == 0) {
      int g = 0;
      for (int i = 0; i < nitems && !*fail; ++i) {
        const Item it = item(p, (int)blockIdx.x + i * (int)gridDim.x);
        const int b = i & 1, v = i >> 1;
        if (v >= 1 && !poll1(tempty(b), (v - 1) & 1, fail)) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t id = idesc(it.npad);
        const uint32_t bterm = TC_KC * it.npad * 16, b_lbo = (uint32_t)it.npad * 16;
        const uint32_t d = tmem + (uint32_t)(b * TC_GMAX);
        bool ok = true;
        for (int kt = 0; kt < p.nk; ++kt, ++g) {
          const int s = g % NS, u = g / NS;
          if (!poll1(afull(s), u & 1, fail) || !poll1(bfull(s), u & 1, fail)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t aHi = s_addr(smem + OFF_A + s * A_STAGE), aLo = aHi + A_TILE;
          const uint32_t bHi = s_addr(smem + OFF_B + s * B_STAGE), bLo = bHi + bterm;
          const int nkk = min(TC_KT / 16, (p.K - kt * TC_KT + 15) / 16);
          for (int kk = 0; kk < nkk; ++kk) {
            const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
            const uint64_t ah = sdesc(aHi + kk * 2 * A_LBO, A_LBO, 128);
            const uint64_t bh = sdesc(bHi + kk * 2 * b_lbo, b_lbo, 128);
            mma(d, ah, bh, id, acc);
            if (p.terms >= 2) mma(d, sdesc(aLo + kk * 2 * A_LBO, A_LBO, 128), bh, id, 1u);
            if (p.terms >= 3) mma(d, ah, sdesc(bLo + kk * 2 * b_lbo, b_lbo, 128), id, 1u);
          }
          commit(sfree(s));
        }
        if (!ok) break;
        commit(tfull(b));
      }
      // every MMA issued above has completed before the tensor memory is freed
      commit(drain);
      poll1(drain, 0, fail);
    }
    __syncwarp();
  } else if (warp >= EPI_WARPS) {
    // ---- converters: warp cw copies rows 16 cw .. 16 cw + 15 of each stage into the FP32
    // ring (each cp.async instruction of the warp covers whole 128-byte row segments:
    // coalesced) and converts them: lane l takes row 16 cw + l % 16, k half l / 16 ----
    const int cw = warp - EPI_WARPS;
    const uint32_t ring = s_addr(smem + OFF_D);
    const int r = 16 * cw + (lane & 15), hk = lane >> 4;  // this thread's tile row and k half
    const int sw = r & 7;  // 16-byte chunk swizzle of a row (conflict-free row reads)
    float tacc[TC_TAILMAX];
#pragma unroll
    for (int c = 0; c < TC_TAILMAX; ++c) tacc[c] = 0.f;
    // issue the copies of stage q (work item q / nk, K stage q % nk) into ring slot q % ND
    auto issue = [&](int q) {
      if (q < nstages) {
        const Item it = item(p, (int)blockIdx.x + (q / p.nk) * (int)gridDim.x);
        const int k0 = (q % p.nk) * TC_KT;
        const uint32_t slot = ring + (uint32_t)((q % ND) * D_STAGE);
#pragma unroll
        for (int c = 0; c < 64 / VEC; ++c) {
          const int o = (c * 32 + lane) * VEC;             // byte within the warp's 16 x 128 B
          const int rr = 16 * cw + (o >> 7), bb = o & 127;  // tile row, byte within its segment
          const int row = it.m0 + rr, k = k0 + (bb >> 2);
          const bool valid = row < p.M_total && k < p.K;
          const float* src = valid ? p.in + (int64_t)row * p.ldin + k : p.in;
          cp_async<VEC>(slot + (uint32_t)(rr * 128 + (((bb >> 4) ^ (rr & 7)) << 4) + (bb & 15)), src,
                        valid ? VEC : 0);
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
    for (int q = 0; q < ND; ++q) issue(q);
    for (int g = 0; g < nstages; ++g) {
      const int s = g % NS, u = g / NS, kt = g % p.nk;
      asm volatile("cp.async.wait_group %0;" ::"n"(ND - 1) : "memory");
      __syncwarp();  // the warp's rows, copied by all of its lanes, are visible to each lane
      if (u >= 1 && !pollw(sfree(s), (u - 1) & 1, fail, lane)) break;
      const uint8_t* dslot = smem + OFF_D + (size_t)(g % ND) * D_STAGE + (size_t)r * 128;
      uint8_t* sA = smem + OFF_A + s * A_STAGE;
      const int k0 = kt * TC_KT;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int kg = 2 * hk + e;
        const float4 a = *(const float4*)(dslot + (((2 * kg) ^ sw) << 4));
        const float4 b = *(const float4*)(dslot + (((2 * kg + 1) ^ sw) << 4));
        uint4 hi, lo;
        split8(a, b, hi, lo);
        const int off = kg * A_LBO + (r >> 3) * 128 + (r & 7) * 16;
        *(uint4*)(sA + off) = hi;
        *(uint4*)(sA + A_TILE + off) = lo;
        if (TAIL && p.tail) {
#pragma unroll
          for (int c = 0; c < TC_TAILMAX; ++c) {
            if (c < p.tail) {
              const float4 w0 = *(const float4*)(sBt + c * TAIL_LD + k0 + 8 * kg);
              const float4 w1 = *(const float4*)(sBt + c * TAIL_LD + k0 + 8 * kg + 4);
              float acc = tacc[c];
              acc = fmaf(a.x, w0.x, acc);
              acc = fmaf(a.y, w0.y, acc);
              acc = fmaf(a.z, w0.z, acc);
              acc = fmaf(a.w, w0.w, acc);
              acc = fmaf(b.x, w1.x, acc);
              acc = fmaf(b.y, w1.y, acc);
              acc = fmaf(b.z, w1.z, acc);
              acc = fmaf(b.w, w1.w, acc);
              tacc[c] = acc;
            }
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(afull(s)) : "memory");
      issue(g + ND);
      if (TAIL && p.tail && kt == p.nk - 1) {
        // the two k halves of a row are in lanes l and l + 16
#pragma unroll
        for (int c = 0; c < TC_TAILMAX; ++c) tacc[c] += __shfl_xor_sync(0xffffffffu, tacc[c], 16);
        const Item it = item(p, (int)blockIdx.x + (g / p.nk) * (int)gridDim.x);
        const int row = it.m0 + r;
        if (hk == 0 && row < p.M_total) {
          const int plane = row / p.R, rr = row - plane * p.R;
          float* o = p.transposed ? p.out + (int64_t)plane * p.ldo * p.P + rr + (int64_t)TC_GMAX * p.ldo
                                  : p.out + (int64_t)row * p.ldo + TC_GMAX;
          const int64_t cs = p.transposed ? p.ldo : 1;
#pragma unroll
          for (int c = 0; c < TC_TAILMAX; ++c)
            if (c < p.tail) o[c * cs] = tacc[c];
        }
#pragma unroll
        for (int c = 0; c < TC_TAILMAX; ++c) tacc[c] = 0.f;
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else {
    // ---- epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (tile rows) and the
    // 16-column chunks of parity w / 4 ----
    const int q = warp & 3, h = warp >> 2;
    float* stg = (float*)(smem + OFF_S) + warp * STG_FLOATS;
    for (int i = 0; i < nitems; ++i) {
      const Item it = item(p, (int)blockIdx.x + i * (int)gridDim.x);
      const int b = i & 1, v = i >> 1;
      if (!pollw(tfull(b), v & 1, fail, lane)) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int row0 = it.m0 + 32 * q;
      const int row = row0 + lane;
      const bool live = row < p.M_total;
      const int nrows = min(32, p.M_total - row0);
      const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * TC_GMAX);
      int64_t obase = 0;
      if (p.transposed) {
        const int plane = row / p.R, rr = row - plane * p.R;
        obase = (int64_t)plane * p.ldo * p.P + rr;
      }
      // the tensor-memory load of the next chunk is in flight while a chunk is stored;
      // a chunk goes through the warp's staging area so that each store instruction writes
      // p.vec consecutive floats per lane (4 or 2 where the output pitch allows it)
      auto store = [&](const uint32_t(&v16)[EPI_COLS], int cc) {
        const int ncol = min(EPI_COLS, it.pc - cc);
        const int64_t col0 = it.c0 + cc;
        if (p.transposed) {
          if (p.vec == 1) {
            if (live) {
              float* o = p.out + obase + col0 * p.ldo;
#pragma unroll
              for (int j = 0; j < EPI_COLS; ++j)
                if (j < ncol) o[(int64_t)j * p.ldo] = __uint_as_float(v16[j]);
            }
            return;
          }
          // staged as [column][row]; a lane then stores vec consecutive rows of one column
          // (rows of a plane are consecutive in the output; R % vec == 0 keeps them in one)
#pragma unroll
          for (int j = 0; j < EPI_COLS; ++j) stg[j * STG_TLD + lane] = __uint_as_float(v16[j]);
          __syncwarp();
          if (p.vec == 4) {
#pragma unroll
            for (int i = 0; i < EPI_COLS / 4; ++i) {
              const int j = 4 * i + (lane >> 3), a = 4 * (lane & 7), rw = row0 + a;
              if (j < ncol && rw < p.M_total) {
                const int plane = rw / p.R, rr = rw - plane * p.R;
                *(float4*)(p.out + (int64_t)plane * p.ldo * p.P + (col0 + j) * p.ldo + rr) =
                    *(const float4*)(stg + j * STG_TLD + a);
              }
            }
          } else {
#pragma unroll
            for (int i = 0; i < EPI_COLS / 2; ++i) {
              const int j = 2 * i + (lane >> 4), a = 2 * (lane & 15), rw = row0 + a;
              if (j < ncol && rw < p.M_total) {
                const int plane = rw / p.R, rr = rw - plane * p.R;
                *(float2*)(p.out + (int64_t)plane * p.ldo * p.P + (col0 + j) * p.ldo + rr) =
                    *(const float2*)(stg + j * STG_TLD + a);
              }
            }
          }
          __syncwarp();
        } else {
          // staged as [row][column], 4-float chunks swizzled by row (c4 ^ (row & 3))
#pragma unroll
          for (int c4 = 0; c4 < EPI_COLS / 4; ++c4)
            *(float4*)(stg + lane * EPI_COLS + ((c4 ^ (lane & 3)) << 2)) =
                make_float4(__uint_as_float(v16[4 * c4]), __uint_as_float(v16[4 * c4 + 1]),
                            __uint_as_float(v16[4 * c4 + 2]), __uint_as_float(v16[4 * c4 + 3]));
          __syncwarp();
          if (p.vec == 4) {
#pragma unroll
            for (int i = 0; i < 32 / 8; ++i) {
              const int rr = 8 * i + (lane >> 2), c4 = lane & 3;
              if (rr < nrows && 4 * c4 < ncol)
                *(float4*)(p.out + (int64_t)(row0 + rr) * p.ldo + col0 + 4 * c4) =
                    *(const float4*)(stg + rr * EPI_COLS + ((c4 ^ (rr & 3)) << 2));
            }
          } else if (p.vec == 2) {
#pragma unroll
            for (int i = 0; i < 32 / 4; ++i) {
              const int rr = 4 * i + (lane >> 3), c2 = lane & 7;
              if (rr < nrows && 2 * c2 < ncol)
                *(float2*)(p.out + (int64_t)(row0 + rr) * p.ldo + col0 + 2 * c2) =
                    *(const float2*)(stg + rr * EPI_COLS + (((c2 >> 1) ^ (rr & 3)) << 2) + 2 * (c2 & 1));
            }
          } else {
            const int cl = lane & 15, rh = lane >> 4;
            if (cl < ncol) {
              float* o = p.out + (int64_t)row0 * p.ldo + col0 + cl;
              for (int rr = rh; rr < nrows; rr += 2)
                o[(int64_t)rr * p.ldo] = stg[rr * EPI_COLS + (((cl >> 2) ^ (rr & 3)) << 2) + (cl & 3)];
            }
          }
          __syncwarp();
        }
      };
      uint32_t ra[EPI_COLS], rb[EPI_COLS];
      int cc = EPI_COLS * h;
      if (cc < it.npad) {
        tmem_ld16(taddr + (uint32_t)cc, ra);
        tmem_wait();
      }
      for (; cc < it.npad; cc += 4 * EPI_COLS) {
        const int c1 = cc + 2 * EPI_COLS, c2 = cc + 4 * EPI_COLS;
        if (c1 < it.npad) tmem_ld16(taddr + (uint32_t)c1, rb);
        store(ra, cc);
        if (c1 < it.npad) {
          tmem_wait();
          if (c2 < it.npad) tmem_ld16(taddr + (uint32_t)c2, ra);
          store(rb, c1);
          if (c2 < it.npad) tmem_wait();
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tempty(b)) : "memory");
    }
  }

  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (tid == 0 && *fail) atomicExch(p.err, 1);
  if (warp == W_MMA) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

uint16_t to_bf16(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;
  u += 0x7fffu + ((u >> 16) & 1u);  // round to nearest even
  return (uint16_t)(u >> 16);
}

float from_bf16(uint16_t b) {
  const uint32_t u = (uint32_t)b << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

int tc_nk_(int K) { return (K + TC_KT - 1) / TC_KT; }
// Output columns beyond the first 256 accumulated in FP32 by the converter threads (a few
// only, square bases K = P; more take a second tensor-core column group).
int tc_tail(int P, int K) { return (P > TC_GMAX && P - TC_GMAX <= TC_TAILMAX && K <= TC_GMAX + TC_TAILMAX) ? P - TC_GMAX : 0; }
int tc_groups(int P, int K) { return tc_tail(P, K) ? 1 : (P + TC_GMAX - 1) / TC_GMAX; }
int tc_gcols(int P, int K) {
  return tc_tail(P, K) ? TC_GMAX : round16((P + tc_groups(P, K) - 1) / tc_groups(P, K));
}
// Bytes of the tensor-core basis tiles (the tail basis, FP32 rows, follows them).
size_t tc_tile_bytes(int P, int K) {
  return (size_t)tc_groups(P, K) * tc_nk_(K) * 2 * TC_KC * tc_gcols(P, K) * 16;
}

}  // namespace

int tc_npad(int P) { return round16(P < 16 ? 16 : P); }

int tc_nk(int K) { return (K + TC_KT - 1) / TC_KT; }

// Basis B (P x K, row-major, FP64) as BF16 hi/lo tiles in the kernel's shared-memory
// layout, per column group g (columns [g G, g G + G), G = tc_gcols(P), rows padded to a
// multiple of 16): stage kt, term, core-matrix column kc, row n: 16 bytes at
// ((kt * 2 + term) * 4 + kc) * npad_g * 16 + n * 16; then the tail rows in FP32.
void tc_prepare_basis(const std::vector<double>& B, int P, int K, std::vector<uint8_t>& out) {
  const int nk = tc_nk(K), ng = tc_groups(P, K), G = tc_gcols(P, K), T = tc_tail(P, K);
  const size_t tiles = tc_tile_bytes(P, K);
  out.assign(tiles + (size_t)T * K * sizeof(float), 0);
  for (int c = 0; c < T; ++c)
    for (int k = 0; k < K; ++k) {
      const float w = (float)B[(size_t)(TC_GMAX + c) * K + k];
      std::memcpy(out.data() + tiles + ((size_t)c * K + k) * sizeof(float), &w, sizeof(float));
    }
  for (int grp = 0; grp < ng; ++grp) {
    const int c0 = grp * G, pc = std::min(G, P - c0), npad = round16(pc);
    uint8_t* gbase = out.data() + (size_t)grp * nk * 2 * TC_KC * G * 16;
    for (int kt = 0; kt < nk; ++kt)
      for (int n = 0; n < npad; ++n)
        for (int kl = 0; kl < TC_KT; ++kl) {
          const int k = kt * TC_KT + kl;
          const double w = (n < pc && k < K) ? B[(size_t)(c0 + n) * K + k] : 0.0;
          const uint16_t hi = to_bf16((float)w);
          const uint16_t lo = to_bf16((float)(w - (double)from_bf16(hi)));
          const int kc = kl / 8, e = kl % 8;
          const size_t off_hi = ((size_t)(kt * 2 + 0) * TC_KC + kc) * npad * 16 + (size_t)n * 16 + e * 2;
          const size_t off_lo = ((size_t)(kt * 2 + 1) * TC_KC + kc) * npad * 16 + (size_t)n * 16 + e * 2;
          std::memcpy(gbase + off_hi, &hi, 2);
          std::memcpy(gbase + off_lo, &lo, 2);
        }
  }
}

// Largest axis length the tensor-core transform takes (two column groups of 256).
int tc_max_axis() { return 2 * TC_GMAX; }

namespace {
template <int VEC>
int set_smem() {
  return cudaFuncSetAttribute(xform_tc_kernel<VEC, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES) !=
             cudaSuccess ||
         cudaFuncSetAttribute(xform_tc_kernel<VEC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES) !=
             cudaSuccess;
}
template <int VEC>
void launch_vec(const TcArgs& a, unsigned grid, cudaStream_t s) {
  if (a.tail)
    xform_tc_kernel<VEC, true><<<grid, TC_THREADS, SMEM_BYTES, s>>>(a);
  else
    xform_tc_kernel<VEC, false><<<grid, TC_THREADS, SMEM_BYTES, s>>>(a);
}
}  // namespace

int tc_configure() {
  static int done = 0;
  if (done) return HELM6_OK;
  if (set_smem<16>() || set_smem<8>() || set_smem<4>()) return HELM6_ERR_CUDA;
  done = 1;
  return HELM6_OK;
}

void launch_xform_tc(const float* in, float* out, const uint8_t* W, int M_total, int K, int P, int terms,
                     int transposed, int R, int* err, cudaStream_t s, int ldin, int ldo) {
  TcArgs a;
  a.in = in;
  a.out = out;
  a.W = W;
  a.M_total = M_total;
  a.K = K;
  a.P = P;
  a.nk = tc_nk(K);
  a.terms = terms;
  a.transposed = transposed;
  a.R = R;
  a.ldin = ldin > 0 ? ldin : K;
  a.ldo = ldo > 0 ? ldo : (transposed ? R : P);
  a.ngroups = tc_groups(P, K);
  a.gcols = tc_gcols(P, K);
  a.tail = tc_tail(P, K);
  a.Bt = a.tail ? (const float*)(W + tc_tile_bytes(P, K)) : nullptr;
  a.nwork = ((M_total + TC_M - 1) / TC_M) * a.ngroups;
  a.err = err;
  {
    // transposed: a lane stores vec consecutive rows of a column (R % vec == 0, so they
    // stay in one plane); row-major: vec consecutive columns (P % vec == 0); both need
    // the output aligned to vec floats
    // (measured: the staged vector stores pay for the row-major output with a pitch that is
    // a multiple of 4, not for the transposed one, whose scalar stores are coalesced already)
    const uintptr_t oa = (uintptr_t)out;
    a.vec = (!transposed && a.ldo % 4 == 0 && oa % 16 == 0) ? 4 : 1;
    if (!transposed && a.ngroups > 1 && (a.gcols % a.vec)) a.vec = 1;
  }
  if (a.nwork == 0) return;
  static int sms = 0;
  if (!sms) sms = device_sm_count();
  const unsigned grid = (unsigned)std::min(a.nwork, sms);
  note_launch();
  const uintptr_t ia = (uintptr_t)in;
  if (a.ldin % 4 == 0 && ia % 16 == 0)
    launch_vec<16>(a, grid, s);
  else if (a.ldin % 2 == 0 && ia % 8 == 0)
    launch_vec<8>(a, grid, s);
  else
    launch_vec<4>(a, grid, s);
}

}  // namespace helm6
