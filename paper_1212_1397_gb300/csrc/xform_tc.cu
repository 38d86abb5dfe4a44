// x/y eigen-transforms of the preconditioner (Eq. 3DAP) on the 5th-generation tensor cores.
//
// One transform contracts every row of a planar FP32 field along its contiguous axis with
// the real basis matrix B (P modes x K points):  out(row, p) = sum_k in(row, k) B(p, k).
// It is a GEMM  D[M x N] = A[M x K] B[N x K]^T  with A = data rows (K-major) and B = basis
// (K-major).  Split precision: each FP32 value x is written to shared memory as BF16
// hi = bf16(x) and lo = bf16(x - hi); the basis is split the same way on the host, and
// D accumulates hi*hi + lo*hi (+ hi*lo) in FP32 in tensor memory (1, 2 or 3 products).
//
// CTA = 128 data rows (one UMMA M) x all N modes.  K is streamed in 64-element stages
// (one 128-byte swizzle row of BF16), double-buffered: the basis stage arrives by a bulk
// copy completing on an mbarrier; the data stage is loaded, split and stored swizzled by
// all threads; one thread issues the MMAs and commits them to a second mbarrier that
// releases the stage.  Every mbarrier wait is bounded; a timeout sets *err, skips the
// remaining work, and the CTA still frees its tensor memory.
//
// Epilogue: each warp reads its 32 tensor-memory lanes (rows) and half of the columns and
// stores either row-major (out[row*P + p]) or transposed within planes of R rows
// (out[(row/R)*R*P + p*R + row%R]), which keeps consecutive lanes on consecutive addresses.
#include <cuda_bf16.h>

#include <cstring>

#include "helm6_internal.h"

namespace helm6 {

namespace {

constexpr int TC_M = 128;
constexpr int TC_KT = 64;
constexpr int TC_THREADS = 256;
constexpr int A_TILE = TC_M * TC_KT * 2;  // bytes of one BF16 term of the data stage
constexpr int kMaxPolls = 1 << 22;

struct TcArgs {
  const float* in;
  float* out;
  const uint8_t* W;  // [kt][term][Npad rows][128 B] pre-swizzled
  int M_total, K, P, Npad, nk, terms, transposed, R;
  int* err;
};

__device__ __forceinline__ uint32_t s_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
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

constexpr int A_PER_THREAD = TC_M * TC_KT / 2 / TC_THREADS;  // float pairs per thread per stage

// Load the FP32 data of stage kt (rows m0.., k in [64 kt, 64 kt + 64)) into registers;
// zero outside the field.  Pairs are 8-byte aligned when K is even.
__device__ __forceinline__ void load_stage(const TcArgs& p, int m0, int kt, int tid, float2* xr) {
  const int kp = (tid & 31) * 2;
  const int k = kt * TC_KT + kp;
#pragma unroll
  for (int i = 0; i < A_PER_THREAD; ++i) {
    const int row = m0 + (tid >> 5) + 8 * i;
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

// Split the stage into BF16 hi / lo and store both in the 128-byte-swizzled K-major layout.
__device__ __forceinline__ void store_stage(uint8_t* sA, int tid, const float2* xr) {
  const int kp = (tid & 31) * 2;
#pragma unroll
  for (int i = 0; i < A_PER_THREAD; ++i) {
    const int r = (tid >> 5) + 8 * i;
    const __nv_bfloat16 h0 = __float2bfloat16_rn(xr[i].x), h1 = __float2bfloat16_rn(xr[i].y);
    const __nv_bfloat16 l0 = __float2bfloat16_rn(xr[i].x - __bfloat162float(h0));
    const __nv_bfloat16 l1 = __float2bfloat16_rn(xr[i].y - __bfloat162float(h1));
    const int off = r * 128 + ((((kp >> 3) ^ (r & 7)) << 4)) + (kp & 7) * 2;
    __nv_bfloat162 hh, ll;
    hh.x = h0;
    hh.y = h1;
    ll.x = l0;
    ll.y = l1;
    *(__nv_bfloat162*)(sA + off) = hh;
    *(__nv_bfloat162*)(sA + A_TILE + off) = ll;
  }
}

__global__ void __launch_bounds__(TC_THREADS, 1) xform_tc_kernel(TcArgs p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int bstage = 2 * p.Npad * 128;  // basis bytes per stage (hi, lo)
  const int stage_bytes = 2 * A_TILE + bstage;
  uint64_t* bars = (uint64_t*)(smem + 2 * stage_bytes);  // full[0..1], done[0..1]
  uint32_t* tslot = (uint32_t*)(bars + 4);
  int* fail = (int*)(tslot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * TC_M;
  const uint32_t ncols = p.Npad > 256 ? 512u : (p.Npad > 128 ? 256u : (p.Npad > 64 ? 128u : (p.Npad > 32 ? 64u : 32u)));
  const uint32_t bar0 = s_addr(bars);
  auto full = [&](int s) { return bar0 + 8u * s; };
  auto done = [&](int s) { return bar0 + 16u + 8u * s; };

  if (tid == 0) {
    for (int s = 0; s < 4; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar0 + 8u * s), "r"(1));
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

  const int btx = (p.terms == 3 ? 2 : 1) * p.Npad * 128;  // bytes the bulk copy brings
  const int nchunk = p.Npad > 256 ? 2 : 1;

  // basis stages 0 and 1 are requested up front; stage kt + 1 is requested as soon as the
  // MMAs of step kt - 1 have released its buffer (right after step kt is committed)
  auto issue_b = [&](int kt) {
    const int st = kt & 1;
    uint8_t* sB = smem + st * stage_bytes + 2 * A_TILE;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(full(st)), "r"(btx) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(s_addr(sB)),
        "l"(p.W + (size_t)kt * bstage), "r"(btx), "r"(full(st))
        : "memory");
  };
  if (tid == 0) {
    issue_b(0);
    if (p.nk > 1) issue_b(1);
  }
  // data stage in registers: thread t holds rows (t >> 5) + 8 i, k pair (t & 31) * 2
  float2 xr[A_PER_THREAD];
  load_stage(p, m0, 0, tid, xr);

  for (int kt = 0; kt < p.nk; ++kt) {
    const int st = kt & 1;
    uint8_t* sA = smem + st * stage_bytes;
    uint8_t* sB = sA + 2 * A_TILE;
    if (kt >= 2 && !*fail) {
      if (!poll(done(st), ((kt - 2) >> 1) & 1)) *fail = 1;
    }
    __syncthreads();
    if (*fail) break;
    store_stage(sA, tid, xr);
    if (kt + 1 < p.nk) load_stage(p, m0, kt + 1, tid, xr);  // in flight during the MMAs
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      if (!poll(full(st), (kt >> 1) & 1)) {
        *fail = 1;
      } else {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t aHi = s_addr(sA), aLo = aHi + A_TILE, bHi = s_addr(sB), bLo = bHi + p.Npad * 128;
#pragma unroll
        for (int kk = 0; kk < TC_KT / 16; ++kk) {
          for (int c = 0; c < nchunk; ++c) {
            const int n0 = c * 128;
            const int nc = (nchunk == 1) ? p.Npad : (c == 0 ? 128 : p.Npad - 128);
            const uint32_t id = idesc(nc);
            const uint32_t t = tmem + (uint32_t)n0;
            const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
            const uint64_t ah = sdesc(aHi + kk * 32), bh = sdesc(bHi + n0 * 128 + kk * 32);
            mma(t, ah, bh, id, acc);
            if (p.terms >= 2) mma(t, sdesc(aLo + kk * 32), bh, id, 1u);
            if (p.terms >= 3) mma(t, ah, sdesc(bLo + n0 * 128 + kk * 32), id, 1u);
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(done(st))
                     : "memory");
        // stage (kt + 1) & 1 was last read by the MMAs of step kt - 1
        if (kt >= 1 && kt + 1 < p.nk) {
          if (!poll(done(st ^ 1), ((kt - 1) >> 1) & 1))
            *fail = 1;
          else
            issue_b(kt + 1);
        }
      }
    }
  }

  // wait for the last committed stage (commits complete in order)
  __syncthreads();
  if (!*fail) {
    const int last = p.nk - 1;
    if (!poll(done(last & 1), (last >> 1) & 1)) *fail = 1;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (!*fail) {
    const int g = warp & 3, h = warp >> 2;
    const int half = p.Npad / 2;
    const int r = 32 * g + lane;  // row within the tile = tensor-memory lane
    const int row = m0 + r;
    const bool live = row < p.M_total;
    // row-major output goes through shared memory (stride P + 1) so that the tile, one
    // contiguous chunk of rows * P floats in global memory, is written coalesced
    float* stile = (float*)smem;
    const int sld = p.P + 1;
    int64_t obase = 0;
    if (p.transposed) {
      const int plane = row / p.R, rr = row - plane * p.R;
      obase = (int64_t)plane * p.R * p.P + rr;
    }
    for (int c0 = h * half; c0 < (h + 1) * half; c0 += 8) {
      uint32_t v[8];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
          : "r"(tmem + ((uint32_t)(32 * g) << 16) + (uint32_t)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int col = c0 + j;
        if (col >= p.P) continue;
        if (p.transposed) {
          if (live) p.out[obase + (int64_t)col * p.R] = __uint_as_float(v[j]);
        } else {
          stile[r * sld + col] = __uint_as_float(v[j]);
        }
      }
    }
    if (!p.transposed) {
      __syncthreads();
      const int rows = min(TC_M, p.M_total - m0);
      float* dst = p.out + (int64_t)m0 * p.P;
      if ((p.P & 3) == 0) {
        // rows of P floats, 16-byte aligned: one warp per row, float4 stores
        const int q4 = p.P >> 2;
        for (int rr = warp; rr < rows; rr += TC_THREADS / 32) {
          const float* srow = stile + rr * sld;
          float4* drow = (float4*)(dst + (int64_t)rr * p.P);
          for (int c4 = lane; c4 < q4; c4 += 32)
            drow[c4] = make_float4(srow[4 * c4], srow[4 * c4 + 1], srow[4 * c4 + 2], srow[4 * c4 + 3]);
        }
      } else {
        for (int rr = warp; rr < rows; rr += TC_THREADS / 32) {
          const float* srow = stile + rr * sld;
          float* drow = dst + (int64_t)rr * p.P;
          for (int cc = lane; cc < p.P; cc += 32) drow[cc] = srow[cc];
        }
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

}  // namespace

int tc_npad(int P) {
  int n = ((P + 15) / 16) * 16;
  return n < 16 ? 16 : n;
}

int tc_nk(int K) { return (K + TC_KT - 1) / TC_KT; }

size_t tc_smem_bytes(int Npad) { return 2 * (size_t)(2 * A_TILE + 2 * Npad * 128) + 64 + 1024; }

// Basis B (P x K, row-major, FP64) as BF16 hi/lo tiles in the swizzled K-major layout the
// kernel's shared memory uses: tile (kt, term) holds rows n < Npad, k in [64 kt, 64 kt+64).
void tc_prepare_basis(const std::vector<double>& B, int P, int K, std::vector<uint8_t>& out) {
  const int Npad = tc_npad(P), nk = tc_nk(K);
  out.assign((size_t)nk * 2 * Npad * 128, 0);
  for (int kt = 0; kt < nk; ++kt) {
    for (int n = 0; n < Npad; ++n) {
      for (int kl = 0; kl < TC_KT; ++kl) {
        const int k = kt * TC_KT + kl;
        double w = (n < P && k < K) ? B[(size_t)n * K + k] : 0.0;
        const uint16_t hi = to_bf16((float)w);
        const uint16_t lo = to_bf16((float)(w - (double)from_bf16(hi)));
        const size_t off = (size_t)n * 128 + ((((kl >> 3) ^ (n & 7)) << 4)) + (kl & 7) * 2;
        uint8_t* base = out.data() + (size_t)kt * 2 * Npad * 128;
        std::memcpy(base + off, &hi, 2);
        std::memcpy(base + (size_t)Npad * 128 + off, &lo, 2);
      }
    }
  }
}

// Largest axis length the tensor-core transform takes: two stages of data (32 KB) and
// basis (2 x Npad x 128 B) must fit in 227 KB of shared memory.
int tc_max_axis() { return 320; }

int tc_configure() {
  static int done = 0;
  if (done) return HELM6_OK;
  const size_t maxs = tc_smem_bytes(tc_npad(tc_max_axis()));
  if (cudaFuncSetAttribute(xform_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)maxs) != cudaSuccess)
    return HELM6_ERR_CUDA;
  done = 1;
  return HELM6_OK;
}

void launch_xform_tc(const float* in, float* out, const uint8_t* W, int M_total, int K, int P, int terms,
                     int transposed, int R, int* err, cudaStream_t s) {
  TcArgs a;
  a.in = in;
  a.out = out;
  a.W = W;
  a.M_total = M_total;
  a.K = K;
  a.P = P;
  a.Npad = tc_npad(P);
  a.nk = tc_nk(K);
  a.terms = terms;
  a.transposed = transposed;
  a.R = R;
  a.err = err;
  const unsigned grid = (unsigned)((M_total + TC_M - 1) / TC_M);
  note_launch();
  xform_tc_kernel<<<grid, TC_THREADS, tc_smem_bytes(a.Npad), s>>>(a);
}

}  // namespace helm6
