// x/y eigen-transforms of the preconditioner (Eq. 3DAP) on the 5th-generation tensor cores.
//
// One transform contracts every row of a planar FP32 field along its contiguous axis with
// the real basis matrix B (P modes x K points):  out(row, p) = sum_k in(row, k) B(p, k).
// It is a GEMM  D[M x N] = A[M x K] B[N x K]^T  with A = data rows (K-major) and B = basis
// (K-major).  Split precision: each FP32 value x is written to shared memory as BF16
// hi = bf16(x) and lo = bf16(x - hi); the basis is split the same way on the host, and
// D accumulates hi*hi + lo*hi (+ hi*lo) in FP32 in tensor memory (1, 2 or 3 products).
//
// CTA = 128 data rows (one MMA M) x one group of at most 256 output columns (P > 256 is
// cut into two groups, interleaved in the grid so that the two CTAs of a row tile run
// together and share its data in L2).  K is streamed in 32-element stages, double
// buffered, in the no-swizzle K-major layout: a core matrix is 8 rows x 16 bytes stored
// contiguously, core matrices 8 rows apart are 128 B apart and the K direction steps by
// one whole column of core matrices.  The basis stage arrives by a bulk copy completing on
// an mbarrier; the data stage is loaded, split and stored by all threads (each warp writes
// whole core matrices, conflict-free); one thread issues the MMAs and commits them to a
// second mbarrier that releases the stage.  At most 256 tensor-memory columns and about
// 100 KB of shared memory per CTA let two CTAs share an SM.  Every mbarrier wait is
// bounded; a timeout sets *err, skips the remaining work, and the CTA still frees its
// tensor memory.
//
// Epilogue: each warp reads its 32 tensor-memory lanes (rows) and half of the columns and
// stores either transposed within planes of R rows (out[(row/R)*R*P + p*R + row%R], which
// keeps consecutive lanes on consecutive addresses) or row-major (out[row*P + p]) through
// shared memory, 64 rows at a time, so that rows are written coalesced.
#include <cuda_bf16.h>

#include <cstring>

#include "helm6_internal.h"

namespace helm6 {

namespace {

constexpr int TC_M = 128;
constexpr int TC_KT = 32;                   // K per stage
constexpr int TC_KC = TC_KT / 8;            // core-matrix columns per stage
constexpr int TC_THREADS = 256;
constexpr int TC_GMAX = 256;                // output columns of one CTA (MMA N limit)
constexpr int A_TILE = TC_M * TC_KT * 2;    // bytes of one BF16 term of the data stage
constexpr int A_LBO = (TC_M / 8) * 128;     // K step of the data stage (one core-matrix column)
constexpr int kMaxPolls = 1 << 22;

struct TcArgs {
  const float* in;
  float* out;
  const uint8_t* W;  // per column group: [kt][term][kc][Npad_g / 8][8 rows][16 B]
  int M_total, K, P, nk, terms, transposed, R;
  int ngroups, gcols;  // column groups and columns per group (the last may have fewer)
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

__device__ __forceinline__ bool poll(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < kMaxPolls; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred P1;\n mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n"
        " selp.b32 %0, 1, 0, P1;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

constexpr int A_PER_THREAD = TC_M * TC_KT / 2 / TC_THREADS;  // float pairs per thread per stage (8)

// Stage kt of the data: core matrix cm = 8 warp + i holds rows 8 (cm % 16) .. + 7 and
// k = 32 kt + 8 (cm / 16) .. + 7; lane l holds row l / 4 and the k pair 2 (l % 4).  Zero
// outside the field.  Pairs are 8-byte aligned when K is even.
__device__ __forceinline__ void load_stage(const TcArgs& p, int m0, int kt, int warp, int lane, float2* xr) {
  const int r8 = lane >> 2, pr = lane & 3;
#pragma unroll
  for (int i = 0; i < A_PER_THREAD; ++i) {
    const int cm = warp * A_PER_THREAD + i;
    const int row = m0 + 8 * (cm & 15) + r8;
    const int k = kt * TC_KT + 8 * (cm >> 4) + 2 * pr;
    float2 v = make_float2(0.f, 0.f);
    if (row < p.M_total) {
      const float* src = p.in + (int64_t)row * p.K + k;
      if (k + 1 < p.K && !(p.K & 1)) {
        v = __ldg((const float2*)src);
      } else {
        if (k < p.K) v.x = __ldg(src);
        if (k + 1 < p.K) v.y = __ldg(src + 1);
      }
    }
    xr[i] = v;
  }
}

// Split the stage into BF16 hi / lo: core matrix cm at (cm / 16) * A_LBO + (cm % 16) * 128.
__device__ __forceinline__ void store_stage(uint8_t* sA, int warp, int lane, const float2* xr) {
#pragma unroll
  for (int i = 0; i < A_PER_THREAD; ++i) {
    const int cm = warp * A_PER_THREAD + i;
    const int off = (cm >> 4) * A_LBO + (cm & 15) * 128 + lane * 4;
    const __nv_bfloat16 h0 = __float2bfloat16_rn(xr[i].x), h1 = __float2bfloat16_rn(xr[i].y);
    const __nv_bfloat16 l0 = __float2bfloat16_rn(xr[i].x - __bfloat162float(h0));
    const __nv_bfloat16 l1 = __float2bfloat16_rn(xr[i].y - __bfloat162float(h1));
    __nv_bfloat162 hh, ll;
    hh.x = h0;
    hh.y = h1;
    ll.x = l0;
    ll.y = l1;
    *(__nv_bfloat162*)(sA + off) = hh;
    *(__nv_bfloat162*)(sA + A_TILE + off) = ll;
  }
}

__host__ __device__ __forceinline__ int round16(int n) { return ((n + 15) / 16) * 16; }
int tc_nk_(int K) { return (K + TC_KT - 1) / TC_KT; }

__global__ void __launch_bounds__(TC_THREADS, 2) xform_tc_kernel(TcArgs p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int grp = (int)(blockIdx.x % p.ngroups);
  const int m0 = (int)(blockIdx.x / p.ngroups) * TC_M;
  const int c0 = grp * p.gcols;                   // first output column of this CTA
  const int pc = min(p.gcols, p.P - c0);          // its columns
  const int npad = round16(pc);                   // MMA N
  const int gpad = round16(p.gcols);              // N of the groups before the last
  const int bterm = TC_KC * npad * 16;            // basis bytes of one term of one stage
  const int bstage = 2 * bterm;
  const int stage_bytes = 2 * A_TILE + 2 * TC_KC * TC_GMAX * 16;  // fixed stride (largest group)
  uint64_t* bars = (uint64_t*)(smem + 2 * stage_bytes);  // full[0..1], done[0..1], afull[0..1]
  uint32_t* tslot = (uint32_t*)(bars + 6);
  int* fail = (int*)(tslot + 1);
  const uint32_t ncols = npad > 128 ? 256u : (npad > 64 ? 128u : (npad > 32 ? 64u : 32u));
  const uint32_t bar0 = s_addr(bars);
  auto full = [&](int s) { return bar0 + 8u * s; };          // basis stage arrived (bulk copy)
  auto done = [&](int s) { return bar0 + 16u + 8u * s; };    // MMAs of the stage completed
  auto afull = [&](int s) { return bar0 + 32u + 8u * s; };   // every thread stored its data part
  // this group's basis: the groups before it hold nk stages of 2 terms of gpad rows each
  const uint8_t* W = p.W + (size_t)grp * p.nk * 2 * TC_KC * gpad * 16;

  if (tid == 0) {
    for (int s = 0; s < 4; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar0 + 8u * s), "r"(1));
    for (int s = 4; s < 6; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar0 + 8u * s), "r"(TC_THREADS));
    asm volatile("fence.mbarrier_init.release.cluster;");
    asm volatile("fence.proxy.async.shared::cta;");
    *fail = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(tslot)), "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;

  const int btx = (p.terms == 3 ? 2 : 1) * bterm;  // bytes the bulk copy brings

  // basis stages 0 and 1 are requested up front; stage kt + 1 is requested as soon as the
  // MMAs of step kt - 1 have released its buffer (right after step kt is committed)
  auto issue_b = [&](int kt) {
    const int st = kt & 1;
    uint8_t* sB = smem + st * stage_bytes + 2 * A_TILE;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(full(st)), "r"(btx) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(s_addr(sB)),
        "l"(W + (size_t)kt * bstage), "r"(btx), "r"(full(st))
        : "memory");
  };
  if (tid == 0) {
    issue_b(0);
    if (p.nk > 1) issue_b(1);
  }
  float2 xr[A_PER_THREAD];
  load_stage(p, m0, 0, warp, lane, xr);
  const uint32_t id = idesc(npad);

  int last_commit = -1;  // thread 0: the last stage whose MMAs were committed
  // No block-wide barrier in the loop: each thread waits only for the MMAs that last read
  // the stage buffer it is about to overwrite, stores its part of the data stage and
  // arrives on afull; thread 0 alone waits for afull and the basis before issuing.
  for (int kt = 0; kt < p.nk; ++kt) {
    const int st = kt & 1;
    uint8_t* sA = smem + st * stage_bytes;
    uint8_t* sB = sA + 2 * A_TILE;
    if (kt >= 2 && !poll(done(st), ((kt - 2) >> 1) & 1)) {
      *fail = 1;
      break;
    }
    store_stage(sA, warp, lane, xr);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(afull(st)) : "memory");
    if (kt + 1 < p.nk) load_stage(p, m0, kt + 1, warp, lane, xr);  // in flight during the MMAs
    if (tid == 0) {
      if (!poll(afull(st), (kt >> 1) & 1) || !poll(full(st), (kt >> 1) & 1)) {
        *fail = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t aHi = s_addr(sA), aLo = aHi + A_TILE, bHi = s_addr(sB), bLo = bHi + bterm;
      const uint32_t b_lbo = (uint32_t)npad * 16;
#pragma unroll
      for (int kk = 0; kk < TC_KT / 16; ++kk) {
        const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
        const uint64_t ah = sdesc(aHi + kk * 2 * A_LBO, A_LBO, 128);
        const uint64_t bh = sdesc(bHi + kk * 2 * b_lbo, b_lbo, 128);
        mma(tmem, ah, bh, id, acc);
        if (p.terms >= 2) mma(tmem, sdesc(aLo + kk * 2 * A_LBO, A_LBO, 128), bh, id, 1u);
        if (p.terms >= 3) mma(tmem, ah, sdesc(bLo + kk * 2 * b_lbo, b_lbo, 128), id, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(done(st))
                   : "memory");
      last_commit = kt;
      // stage (kt + 1) & 1 was last read by the MMAs of step kt - 1
      if (kt >= 1 && kt + 1 < p.nk) {
        if (!poll(done(st ^ 1), ((kt - 1) >> 1) & 1)) {
          *fail = 1;
          break;
        }
        issue_b(kt + 1);
      }
    }
  }

  // wait for the last committed stage (commits complete in order), also after a timeout
  // elsewhere: no MMA may still write tensor memory when it is freed below
  __syncthreads();
  if (tid == 0 && last_commit >= 0 && !poll(done(last_commit & 1), (last_commit >> 1) & 1)) *fail = 1;
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (!*fail) {
    const int g = warp & 3, h = warp >> 2;
    const int half = ((npad / 8 + 1) / 2) * 8;  // columns of warp half 0 (multiple of 8)
    const int cbeg = h ? half : 0, cend = h ? npad : half;
    const int r = 32 * g + lane;  // row within the tile = tensor-memory lane
    const int row = m0 + r;
    const bool live = row < p.M_total;
    if (p.transposed) {
      const int plane = row / p.R, rr = row - plane * p.R;
      const int64_t obase = (int64_t)plane * p.R * p.P + rr;
      for (int cc = cbeg; cc < cend; cc += 8) {
        uint32_t v[8];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
            : "r"(tmem + ((uint32_t)(32 * g) << 16) + (uint32_t)cc));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (cc + j < pc && live) p.out[obase + (int64_t)(c0 + cc + j) * p.R] = __uint_as_float(v[j]);
      }
    } else {
      // row-major: 64 rows at a time through shared memory (stride pc + 1), then each warp
      // copies whole rows of pc floats to out[row * P + c0 ..]
      float* stile = (float*)smem;
      const int sld = pc + 1;
      for (int pass = 0; pass < 2; ++pass) {
        if ((g >> 1) == pass) {
          const int rl = r - 64 * pass;
          // four 8-column loads per wait (faster here; the transposed path above is not)
          for (int cc = cbeg; cc < cend; cc += 32) {
            uint32_t v[32];
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (cc + 8 * q < cend)
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                    : "=r"(v[8 * q]), "=r"(v[8 * q + 1]), "=r"(v[8 * q + 2]), "=r"(v[8 * q + 3]), "=r"(v[8 * q + 4]),
                      "=r"(v[8 * q + 5]), "=r"(v[8 * q + 6]), "=r"(v[8 * q + 7])
                    : "r"(tmem + ((uint32_t)(32 * g) << 16) + (uint32_t)(cc + 8 * q)));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (cc + j < cend && cc + j < pc) stile[rl * sld + cc + j] = __uint_as_float(v[j]);
          }
        }
        __syncthreads();
        const int rows = min(64, p.M_total - (m0 + 64 * pass));
        float* dst = p.out + (int64_t)(m0 + 64 * pass) * p.P + c0;
        // consecutive lanes on consecutive words: conflict-free reads, 128-byte stores
        for (int rr = warp; rr < rows; rr += TC_THREADS / 32) {
          const float* srow = stile + rr * sld;
          float* drow = dst + (int64_t)rr * p.P;
          for (int cc = lane; cc < pc; cc += 32) drow[cc] = srow[cc];
        }
        __syncthreads();
      }
    }
  } else if (tid == 0) {
    atomicExch(p.err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
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

// Columns beyond the first 256 computed by the FP32 tail kernel (a few only; more take a
// second tensor-core column group).
constexpr int TC_TAILMAX = 32;
constexpr int TC_TAILK = TC_GMAX + TC_TAILMAX;  // longest row on the tail path (square bases: K = P)
int tc_tail(int P, int K) { return (P > TC_GMAX && P - TC_GMAX <= TC_TAILMAX && K <= TC_TAILK) ? P - TC_GMAX : 0; }
int tc_groups(int P, int K) { return tc_tail(P, K) ? 1 : (P + TC_GMAX - 1) / TC_GMAX; }
int tc_gcols(int P, int K) {
  return tc_tail(P, K) ? TC_GMAX : round16((P + tc_groups(P, K) - 1) / tc_groups(P, K));
}
// Bytes of the tensor-core basis tiles (the tail basis, FP32 rows, follows them).
size_t tc_tile_bytes(int P, int K) {
  return (size_t)tc_groups(P, K) * tc_nk_(K) * 2 * TC_KC * tc_gcols(P, K) * 16;
}

// The last P - 256 output columns: out(row, 256 + c) = sum_k in(row, k) Bt(c, k) in FP32, one
// warp per row (lanes stride over k, shuffle reduction), Bt staged in shared memory.  TT > 0:
// that many columns, known at compile time; TT = 0: any T <= TC_TAILMAX.
template <int TT>
__global__ void __launch_bounds__(256) xform_tail_kernel(const float* __restrict__ in, float* __restrict__ out,
                                                         const float* __restrict__ Bt, int M_total, int K, int P,
                                                         int T_rt, int transposed, int R) {
  constexpr int TM = TT > 0 ? TT : TC_TAILMAX;
  const int T = TT > 0 ? TT : T_rt;
  extern __shared__ float sbt[];
  for (int i = threadIdx.x; i < T * K; i += blockDim.x) sbt[i] = Bt[i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t row = (int64_t)blockIdx.x * 8 + warp; row < M_total; row += (int64_t)gridDim.x * 8) {
    const float* r = in + row * K;
    float acc[TM];
#pragma unroll
    for (int c = 0; c < TM; ++c) acc[c] = 0.f;
    // the whole row first (K <= 288 on this path: at most 9 values per lane), so that all
    // of a warp's loads are in flight together
    float v[TC_TAILK / 32];
#pragma unroll
    for (int q = 0; q < TC_TAILK / 32; ++q) {
      const int k = lane + 32 * q;
      v[q] = k < K ? __ldg(r + k) : 0.f;
    }
#pragma unroll
    for (int q = 0; q < TC_TAILK / 32; ++q) {
      const int k = lane + 32 * q;
      if (k >= K) break;
      if constexpr (TT > 0) {
#pragma unroll
        for (int c = 0; c < TT; ++c) acc[c] = fmaf(v[q], sbt[c * K + k], acc[c]);
      } else {
#pragma unroll
        for (int c = 0; c < TM; ++c)
          if (c < T) acc[c] = fmaf(v[q], sbt[c * K + k], acc[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < TM; ++c) {
      if (c >= T) break;
      float x = acc[c];
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == c) {
        const int col = TC_GMAX + c;
        if (transposed) {
          const int64_t plane = row / R, rr = row - plane * R;
          out[plane * R * P + (int64_t)col * R + rr] = x;
        } else {
          out[row * P + col] = x;
        }
      }
    }
  }
}

}  // namespace

int tc_npad(int P) { return round16(P < 16 ? 16 : P); }

int tc_nk(int K) { return (K + TC_KT - 1) / TC_KT; }

// two stages of data (2 x 8 KB) and basis (2 terms x 4 core-matrix columns x 256 rows x 16 B)
size_t tc_smem_bytes(int) { return 2 * (size_t)(2 * A_TILE + 2 * TC_KC * TC_GMAX * 16) + 64 + 1024; }

// Basis B (P x K, row-major, FP64) as BF16 hi/lo tiles in the kernel's shared-memory
// layout, per column group g (columns [g G, g G + G), G = tc_gcols(P), rows padded to a
// multiple of 16): stage kt, term, core-matrix column kc, row n: 16 bytes at
// ((kt * 2 + term) * 4 + kc) * npad_g * 16 + n * 16.
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

int tc_configure() {
  static int done = 0;
  if (done) return HELM6_OK;
  if (cudaFuncSetAttribute(xform_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes(0)) !=
      cudaSuccess)
    return HELM6_ERR_CUDA;
  done = 1;
  return HELM6_OK;
}

void launch_xform_tc(const float* in, float* out, const uint8_t* W, int M_total, int K, int P, int terms,
                     int transposed, int R, int* err, cudaStream_t s, cudaStream_t aux, cudaEvent_t fork,
                     cudaEvent_t join) {
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
  a.ngroups = tc_groups(P, K);
  a.gcols = tc_gcols(P, K);
  a.err = err;
  a.P = P;
  const unsigned grid = (unsigned)(((M_total + TC_M - 1) / TC_M) * a.ngroups);
  const bool side = tc_tail(P, K) > 0 && aux && fork && join;
  if (side) {  // fork before the tensor-core kernel so that the tail can start with it
    cudaEventRecord(fork, s);
    cudaStreamWaitEvent(aux, fork, 0);
  }
  note_launch();
  xform_tc_kernel<<<grid, TC_THREADS, tc_smem_bytes(0), s>>>(a);
  const int T = tc_tail(P, K);
  if (T > 0) {
    static int sms = 0;
    if (!sms) sms = device_sm_count();
    const float* Bt = (const float*)(W + tc_tile_bytes(P, K));
    note_launch();
    const size_t sm = (size_t)T * K * sizeof(float);
    const int g = 8 * sms;
    // with an auxiliary stream the tail runs beside the tensor-core kernel (both only read
    // `in`, and write disjoint columns of `out`); s waits for it before any later work
    cudaStream_t ts = side ? aux : s;
    switch (T) {
      case 1: xform_tail_kernel<1><<<g, 256, sm, ts>>>(in, out, Bt, M_total, K, P, T, transposed, R); break;
      case 2: xform_tail_kernel<2><<<g, 256, sm, ts>>>(in, out, Bt, M_total, K, P, T, transposed, R); break;
      case 3: xform_tail_kernel<3><<<g, 256, sm, ts>>>(in, out, Bt, M_total, K, P, T, transposed, R); break;
      case 4: xform_tail_kernel<4><<<g, 256, sm, ts>>>(in, out, Bt, M_total, K, P, T, transposed, R); break;
      default: xform_tail_kernel<0><<<g, 256, sm, ts>>>(in, out, Bt, M_total, K, P, T, transposed, R); break;
    }
    if (ts != s) {
      cudaEventRecord(join, ts);
      cudaStreamWaitEvent(s, join, 0);
    }
  }
}

}  // namespace helm6
