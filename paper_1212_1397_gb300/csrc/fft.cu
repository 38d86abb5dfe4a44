// Fast x/y transforms of the separable preconditioner (Section 3.3, Eq. 3DAP: the direct
// solver of A_p is "FFT-type"; Section 1: O(N^2 N_z log N) per application).
//
// Each of the four closed-form eigenbases of the 1D second-difference matrix (D-D sine,
// N-N cosine, D-N and N-D quarter-wave) is a sine or cosine sum sum_l x_l trig(pi a l j / N)
// with N = n + 1 intervals.  The basis matrices are real, so a complex line (real plane +
// i * imaginary plane) goes through one complex DFT and both planes are transformed at once.
//
// Extending the line oddly (sine) or evenly (cosine) to the length L = 2N (D-D, N-N) or
// L = 4N (D-N, N-D) turns the sum into one complex DFT of length L,
//     E_j = sum_l e_l w^{l j},  w = exp(-2 pi i / L),
// since sum e_l (w^{lj} - w^{-lj}) = -2i sum e_l sin(2 pi l j / L) for an odd extension and
// 2 sum w_l e_l cos(2 pi l j / L) for an even one.
//
// D-D and N-N take the same extension form (L = 2N) or, in the half-length form, a DFT of
// length L = N.  With s_j = sin(pi j / N), the line
//     y_j = s_j (x_j + x_{N-j}) + (x_j - x_{N-j}) / 2            (sine, x_0 = x_N = 0)
//     y_j = (x_j + x_{N-j}) / 2 - s_j (x_j - x_{N-j})            (cosine, nodes 0..N)
// has DFT Z with A_k = (Z_k + Z_{N-k}) / 2 and B_k = i (Z_k - Z_{N-k}) / 2 such that
//     sine:   S_2k = B_k,  S_2k+1 - S_2k-1 = A_k,  S_1 = A_0 / 2,
//     cosine: C_2k = A_k,  C_2k+1 - C_2k-1 = B_k,  C_1 = sum_j w_j x_j cos(pi j / N)
// (the symmetric part of y carries the cosines of even multiples, the antisymmetric part,
// through 2 sin a sin b = cos(a - b) - cos(a + b), the differences of the odd ones), so the
// odd outputs are a prefix sum over k.  This halves the DFT length of the extension form; the
// library takes it in FP64, where the FP64 pipe bounds the kernel, and keeps the extension
// form in FP32, where its rounding (no prefix sum) costs fewer iterations.
//
// The DFT of length L = P * Q (P a power of two, Q = 1 or an odd prime with Q - 1 a power of
// two, which covers n + 1 = 2^k and the prime n + 1 = 257 of the 256^3 grid) is a
// Cooley-Tukey split: P DFTs of length Q on the stride-P subsequences, twiddles w_L^{l1 j2},
// then Q DFTs of length P.  A DFT of prime length Q is Rader's cyclic convolution of length
// M = Q - 1 over the generator powers g^q, done with two radix-2 FFTs of length M and the
// precomputed spectrum of the kernel w_Q^{g^-q}.  Everything between the load and the store
// runs in shared memory; the DRAM traffic is one read and one write of each line.
#include "helm6_internal.h"

#include <cmath>
#include <cstring>

namespace helm6 {

namespace {

template <typename T>
struct Vec2;
template <>
struct Vec2<double> {
  using t = double2;
};
template <>
struct Vec2<float> {
  using t = float2;
};

template <typename V>
__device__ __forceinline__ V cmul(V a, V b) {
  V r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
// a * conj(b)
template <typename V>
__device__ __forceinline__ V cmulc(V a, V b) {
  V r;
  r.x = a.x * b.x + a.y * b.y;
  r.y = a.y * b.x - a.x * b.y;
  return r;
}

__device__ __forceinline__ int brev(int j, int logn) {
  return logn ? (int)(__brev((unsigned)j) >> (32 - logn)) : 0;
}

// Radix-2 decimation in frequency, in place, on nseq sequences of length 2^logn at base +
// s * stride: natural order in, bit-reversed order out.  tw[k] = w_n^k, k < n/2.
template <typename V>
__device__ void fft_dif(V* base, int nseq, int stride, int logn, const V* tw) {
  if (logn == 0) return;
  const int hmask = (1 << (logn - 1)) - 1, nb = nseq << (logn - 1);
  for (int st = logn - 1; st >= 0; --st) {
    const int half = 1 << st, tsh = logn - 1 - st;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
      const int s = b >> (logn - 1), w = b & hmask;
      const int k = w & (half - 1), grp = w >> st;
      V* x = base + s * stride + (grp << (st + 1)) + k;
      const V u = x[0], v = x[half];
      V a, d;
      a.x = u.x + v.x;
      a.y = u.y + v.y;
      d.x = u.x - v.x;
      d.y = u.y - v.y;
      x[0] = a;
      x[half] = k ? cmul(d, tw[k << tsh]) : d;
    }
    __syncthreads();
  }
}

// Radix-2 decimation in time with conjugate twiddles (the unscaled inverse DFT), in place:
// bit-reversed order in, natural order out.
template <typename V>
__device__ void fft_dit_inv(V* base, int nseq, int stride, int logn, const V* tw) {
  if (logn == 0) return;
  const int hmask = (1 << (logn - 1)) - 1, nb = nseq << (logn - 1);
  for (int st = 0; st < logn; ++st) {
    const int half = 1 << st, tsh = logn - 1 - st;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
      const int s = b >> (logn - 1), w = b & hmask;
      const int k = w & (half - 1), grp = w >> st;
      V* x = base + s * stride + (grp << (st + 1)) + k;
      const V u = x[0];
      const V v = k ? cmulc(x[half], tw[k << tsh]) : x[half];
      V a, d;
      a.x = u.x + v.x;
      a.y = u.y + v.y;
      d.x = u.x - v.x;
      d.y = u.y - v.y;
      x[0] = a;
      x[half] = d;
    }
    __syncthreads();
  }
}

struct FftLines {
  int rows;     // complex lines
  int rdiv;     // line r starts at (r / rdiv) * hi + (r % rdiv) * lo
  int64_t hi, lo;
  int64_t es;   // element stride along a line
  int64_t N;    // offset of the imaginary plane
};

// One CTA transforms B lines.  ALONG: the lines are contiguous (x axis), so consecutive
// threads walk one line; otherwise consecutive threads walk consecutive lines (y axis).
template <typename T, bool ALONG>
__global__ void __launch_bounds__(256) fft_axis_kernel(FftDev f, const T* __restrict__ in, T* __restrict__ out,
                                                       FftLines ln, int B, int inv) {
  using V = typename Vec2<T>::t;
  extern __shared__ __align__(16) unsigned char fsm[];
  const int P = f.P, Q = f.Q, M = f.M, L = f.L, logP = f.logP, logM = f.logM;
  const int hP = P >> 1, hM = M >> 1;
  V* sTwP = reinterpret_cast<V*>(fsm);
  V* sTwM = sTwP + hP;
  V* sBh = sTwM + hM;
  V* sE = sBh + M;
  V* sW = sE + (size_t)B * L;
  V* sAux = sW + (size_t)B * P * M;
  V* sX = sAux + (Q > 1 ? 2 * B * P : 0);  // sine/cosine: the lines by node 0..N
  const bool half = f.half;
  int* sG = reinterpret_cast<int*>(sX + (half ? (size_t)B * (f.N + 1) : 0));
  int* sGi = sG + M;
  const V* gtw = reinterpret_cast<const V*>(sizeof(T) == 8 ? (const void*)f.tw64 : (const void*)f.tw32);
  const V* gTwL = gtw + hP + hM + M;
  const V* gCS = gTwL + (Q > 1 ? L : 0);  // sine/cosine: (cos, sin)(pi j / N), j = 0..N
  const int tid = threadIdx.x, nt = blockDim.x;

  for (int e = tid; e < hP + hM + M; e += nt) sTwP[e] = gtw[e];
  for (int e = tid; e < 2 * M; e += nt) sG[e] = f.gidx[e];

  const int r0 = blockIdx.x * B;
  const int nb = min(B, ln.rows - r0);
  const int m = f.m, N = f.N, kind = f.kind;
  const bool odd = kind == 0 || kind == 2, quarter = kind >= 2;
  const int X1 = N + 1;

  if (half) {
    // load the line by node into sX (sine: x_0 = x_N = 0), then y_j into sE
    if (kind == 0)
      for (int e = tid; e < nb; e += nt) sX[e * X1] = sX[e * X1 + N] = V{T(0), T(0)};
    for (int e = tid; e < nb * m; e += nt) {
      int r, p;
      if (ALONG) {
        r = e / m;
        p = e - r * m;
      } else {
        p = e / nb;
        r = e - p * nb;
      }
      const int gr = r0 + r;
      const int64_t g = (int64_t)(gr / ln.rdiv) * ln.hi + (int64_t)(gr % ln.rdiv) * ln.lo + (int64_t)p * ln.es;
      const int j = p + (kind == 0 ? 1 : 0);
      const T wgt = (kind == 1 && inv && (j == 0 || j == N)) ? T(2) : T(1);
      V x;
      x.x = wgt * in[g];
      x.y = wgt * in[g + ln.N];
      sX[r * X1 + j] = x;
    }
    __syncthreads();
    for (int e = tid; e < nb * N; e += nt) {
      const int r = e / N, j = e - r * N;
      const V a = sX[r * X1 + j], b = sX[r * X1 + N - j];
      const T sn = gCS[j].y;
      V y;
      if (kind == 0) {
        y.x = sn * (a.x + b.x) + T(0.5) * (a.x - b.x);
        y.y = sn * (a.y + b.y) + T(0.5) * (a.y - b.y);
      } else {
        y.x = T(0.5) * (a.x + b.x) - sn * (a.x - b.x);
        y.y = T(0.5) * (a.y + b.y) - sn * (a.y - b.y);
      }
      sE[r * L + j] = y;
    }
    __syncthreads();
  } else {
    for (int e = tid; e < nb * L; e += nt) sE[e] = V{T(0), T(0)};
    __syncthreads();
    // load: stored index p -> extension position pos (and its mirror L - pos)
    for (int e = tid; e < nb * m; e += nt) {
      int r, p;
      if (ALONG) {
        r = e / m;
        p = e - r * m;
      } else {
        p = e / nb;
        r = e - p * nb;
      }
      const int gr = r0 + r;
      const int64_t g = (int64_t)(gr / ln.rdiv) * ln.hi + (int64_t)(gr % ln.rdiv) * ln.lo + (int64_t)p * ln.es;
      T wgt = T(1);
      int pos;
      if (!inv) {
        pos = p + ((kind == 0 || kind == 2) ? 1 : 0);  // node l
        if (kind == 2 && pos == N) wgt = T(0.5);
      } else {
        const int j = p + (kind == 1 ? 0 : 1);  // mode j
        pos = quarter ? 2 * j - 1 : j;
        if (kind == 1 && (j == 0 || j == N)) wgt = T(2);
      }
      V x;
      x.x = wgt * in[g];
      x.y = wgt * in[g + ln.N];
      sE[r * L + pos] = x;
      if (pos != 0 && 2 * pos != L) {
        if (odd) {
          x.x = -x.x;
          x.y = -x.y;
        }
        sE[r * L + L - pos] = x;
      }
    }
    __syncthreads();
  }

  if (Q > 1) {
    // Rader: the DFT of length Q of u_l2 = e_{l1 + P l2} is U_0 = u_0 + sum_q a_q and
    // U_{g^-r} = u_0 + (a * b)_r with a_q = u_{g^q}, b_q = w_Q^{g^-q} (cyclic, length M)
    for (int e = tid; e < nb * P * M; e += nt) {
      const int q = e & (M - 1), s = e >> logM;
      const int r = s >> logP, l1 = s & (P - 1);
      sW[e] = sE[r * L + l1 + P * sG[q]];
    }
    for (int e = tid; e < nb * P; e += nt) sAux[2 * e] = sE[(e >> logP) * L + (e & (P - 1))];
    __syncthreads();
    fft_dif(sW, nb * P, M, logM, sTwM);
    for (int e = tid; e < nb * P * M; e += nt) {
      const int k = e & (M - 1);
      const V a = sW[e];
      if (k == 0) sAux[2 * (e >> logM) + 1] = a;
      sW[e] = cmul(a, sBh[k]);  // the kernel's spectrum / M, stored bit-reversed
    }
    __syncthreads();
    fft_dit_inv(sW, nb * P, M, logM, sTwM);
    // U_j2 times w_L^{l1 j2}, stored at j2 * P + l1 for the length-P DFTs
    for (int e = tid; e < nb * P * M; e += nt) {
      const int rr = e & (M - 1), s = e >> logM;
      const int r = s >> logP, l1 = s & (P - 1);
      const int j2 = sGi[rr];
      const V u0 = sAux[2 * s];
      V v = sW[e];
      v.x += u0.x;
      v.y += u0.y;
      sE[r * L + j2 * P + l1] = l1 ? cmul(v, gTwL[l1 * j2]) : v;
    }
    for (int e = tid; e < nb * P; e += nt) {
      const V u0 = sAux[2 * e], a0 = sAux[2 * e + 1];
      V v;
      v.x = u0.x + a0.x;
      v.y = u0.y + a0.y;
      sE[(e >> logP) * L + (e & (P - 1))] = v;
    }
    __syncthreads();
  }
  // length-P DFTs over contiguous groups (the whole line when Q = 1): E_{Q j1 + j2} ends at
  // j2 * P + bitrev(j1)
  fft_dif(sE, nb * Q, P, logP, sTwP);

  const T invN = T(1) / T(N);
  if (half) {
    // one warp per line: A_k, B_k for k = 0..N/2, the even outputs directly and the odd ones
    // as the base plus a running (warp-scanned) sum of the increments, written by node into sX
    const int lane = tid & 31, nw = nt >> 5, kmax = N / 2;
    for (int r = tid >> 5; r < nb; r += nw) {
      V* X = sX + r * X1;
      const V* E = sE + r * L;
      V carry;
      if (kind == 0) {
        const V z0 = E[0];  // Z_0 sits at position 0 in every split
        carry.x = T(0.5) * z0.x;
        carry.y = T(0.5) * z0.y;
      } else {
        T cx = T(0), cy = T(0);
        for (int j = lane; j <= N; j += 32) {
          const T c = gCS[j].x * ((j == 0 || j == N) ? T(0.5) : T(1));
          cx += c * X[j].x;
          cy += c * X[j].y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          cx += __shfl_xor_sync(0xffffffffu, cx, o);
          cy += __shfl_xor_sync(0xffffffffu, cy, o);
        }
        carry.x = cx;
        carry.y = cy;
      }
      __syncwarp();
      for (int k0 = 0; k0 <= kmax; k0 += 32) {
        const int k = k0 + lane;
        const bool valid = k <= kmax;
        V a{T(0), T(0)}, bb{T(0), T(0)};
        if (valid) {
          const int km = k ? N - k : 0;
          const V zk = E[(k % Q) * P + brev(k / Q, logP)];
          const V zm = E[(km % Q) * P + brev(km / Q, logP)];
          a.x = T(0.5) * (zk.x + zm.x);
          a.y = T(0.5) * (zk.y + zm.y);
          bb.x = T(-0.5) * (zk.y - zm.y);
          bb.y = T(0.5) * (zk.x - zm.x);
        }
        V inc{T(0), T(0)};
        if (valid && k >= 1) inc = (kind == 0) ? a : bb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const T tx = __shfl_up_sync(0xffffffffu, inc.x, o), ty = __shfl_up_sync(0xffffffffu, inc.y, o);
          if (lane >= o) {
            inc.x += tx;
            inc.y += ty;
          }
        }
        if (valid) {
          V od;
          od.x = carry.x + inc.x;
          od.y = carry.y + inc.y;
          if (kind == 0) {
            if (k >= 1 && 2 * k <= N - 1) X[2 * k] = bb;
            if (2 * k + 1 <= N - 1) X[2 * k + 1] = od;
          } else {
            if (2 * k <= N) X[2 * k] = a;
            if (2 * k + 1 <= N) X[2 * k + 1] = od;
          }
        }
        carry.x += __shfl_sync(0xffffffffu, inc.x, 31);
        carry.y += __shfl_sync(0xffffffffu, inc.y, 31);
      }
    }
    __syncthreads();
    // store: sine forward 2/N, cosine forward (2/N) w_j, inverses 1
    for (int e = tid; e < nb * m; e += nt) {
      int r, o;
      if (ALONG) {
        r = e / m;
        o = e - r * m;
      } else {
        o = e / nb;
        r = e - o * nb;
      }
      const int j = o + (kind == 0 ? 1 : 0);
      const T sc = inv ? T(1) : ((kind == 1 && (j == 0 || j == N)) ? invN : T(2) * invN);
      const V v = sX[r * X1 + j];
      const int gr = r0 + r;
      const int64_t g = (int64_t)(gr / ln.rdiv) * ln.hi + (int64_t)(gr % ln.rdiv) * ln.lo + (int64_t)o * ln.es;
      out[g] = sc * v.x;
      out[g + ln.N] = sc * v.y;
    }
    return;
  }

  // extension store: stored index o -> E index and the scale of the transform
  for (int e = tid; e < nb * m; e += nt) {
    int r, o;
    if (ALONG) {
      r = e / m;
      o = e - r * m;
    } else {
      o = e / nb;
      r = e - o * nb;
    }
    int eidx;
    T sc;
    if (!inv) {
      const int j = o + (kind == 1 ? 0 : 1);  // mode j
      eidx = quarter ? 2 * j - 1 : j;
      sc = (kind == 1 && (j == 0 || j == N)) ? T(0.5) * invN : invN;
    } else {
      eidx = o + ((kind == 0 || kind == 2) ? 1 : 0);  // node l
      sc = T(0.5);
    }
    const int j1 = eidx / Q, j2 = eidx - j1 * Q;
    const V v = sE[r * L + j2 * P + brev(j1, logP)];
    const int gr = r0 + r;
    const int64_t g = (int64_t)(gr / ln.rdiv) * ln.hi + (int64_t)(gr % ln.rdiv) * ln.lo + (int64_t)o * ln.es;
    if (odd) {  // i * sc * E
      out[g] = -sc * v.y;
      out[g + ln.N] = sc * v.x;
    } else {
      out[g] = sc * v.x;
      out[g + ln.N] = sc * v.y;
    }
  }
}

// exp(-2 pi i t / L) with the angle reduced to the first quadrant exactly, so that the
// quarter-turn roots come out exact.
void unit_root(int64_t t, int64_t L, double& c, double& s) {
  t %= L;
  if (t < 0) t += L;
  const int64_t q = (4 * t) / L, r = 4 * t - q * L;  // angle = q pi/2 + (pi/2) r / L
  double cc, ss;
  if (2 * r <= L) {
    const double th = (M_PI / 2) * (double)r / (double)L;
    cc = std::cos(th);
    ss = std::sin(th);
  } else {
    const double th = (M_PI / 2) * (double)(L - r) / (double)L;
    cc = std::sin(th);
    ss = std::cos(th);
  }
  switch (q) {
    case 0: c = cc; s = ss; break;
    case 1: c = -ss; s = cc; break;
    case 2: c = -cc; s = -ss; break;
    default: c = ss; s = -cc; break;
  }
  s = -s;
}

bool is_prime(int q) {
  if (q < 2) return false;
  for (int d = 2; (int64_t)d * d <= q; ++d)
    if (q % d == 0) return false;
  return true;
}

int primitive_root(int q) {
  for (int g = 2; g < q; ++g) {
    int64_t x = 1;
    int ord = 0;
    do {
      x = x * g % q;
      ++ord;
    } while (x != 1);
    if (ord == q - 1) return g;
  }
  return 1;  // q = 2 (not used)
}

int ilog2(int x) {
  int l = 0;
  while ((1 << l) < x) ++l;
  return l;
}

size_t smem_of(const FftDev& f, int B, int eb) {
  const size_t V = 2 * (size_t)eb;
  size_t c = (size_t)f.P / 2 + f.M / 2 + f.M + (size_t)B * f.L + (size_t)B * f.P * f.M;
  if (f.Q > 1) c += 2 * (size_t)B * f.P;
  if (f.half) c += (size_t)B * (f.N + 1);
  return c * V + 2 * (size_t)f.M * sizeof(int);
}

constexpr size_t kFftSmemMax = 227 * 1024;

}  // namespace

bool fft_make_plan(int n, int lo, int hi, bool half, FftHostPlan& h) {
  const bool nlo = lo != HELM6_DIRICHLET, nhi = hi != HELM6_DIRICHLET;
  FftDev& f = h.d;
  f = FftDev{};
  f.kind = (!nlo && !nhi) ? 0 : (nlo && nhi) ? 1 : (!nlo) ? 2 : 3;
  f.N = n + 1;
  f.m = n + (nlo ? 1 : 0) + (nhi ? 1 : 0);
  f.half = half && f.kind < 2;
  f.L = f.half ? f.N : (f.kind >= 2 ? 4 : 2) * f.N;
  f.P = 1;
  while (f.L % (2 * f.P) == 0) f.P *= 2;
  f.Q = f.L / f.P;
  if (f.Q > 1) {
    // Rader with a power-of-two convolution; the kernel spectrum is formed directly (M^2)
    if (!is_prime(f.Q) || ((f.Q - 1) & (f.Q - 2)) != 0 || f.Q > 257) return false;
    f.M = f.Q - 1;
  }
  f.logP = ilog2(f.P);
  f.logM = f.M ? ilog2(f.M) : 0;
  if (smem_of(f, 1, 8) > kFftSmemMax) return false;

  // complex tables, interleaved: [w_P^k: P/2][w_M^k: M/2][bhat: M][w_L^t: L when Q > 1]
  // [(cos, sin)(pi j / N), j = 0..N: sine and cosine axes]
  const int nt = f.P / 2 + f.M / 2 + f.M + (f.Q > 1 ? f.L : 0) + (f.half ? f.N + 1 : 0);
  h.tw.assign(2 * (size_t)nt, 0.0);
  double* t = h.tw.data();
  for (int k = 0; k < f.P / 2; ++k, t += 2) unit_root(k, f.P, t[0], t[1]);
  for (int k = 0; k < f.M / 2; ++k, t += 2) unit_root(k, f.M, t[0], t[1]);
  h.gidx.assign(2 * (size_t)f.M, 0);
  if (f.Q > 1) {
    const int g = primitive_root(f.Q);
    int64_t x = 1;
    for (int q = 0; q < f.M; ++q, x = x * g % f.Q) h.gidx[q] = (int)x;  // g^q
    for (int r = 0; r < f.M; ++r) h.gidx[f.M + r] = h.gidx[(f.M - r) % f.M];  // g^-r
    // spectrum of b_q = w_Q^{g^-q}, divided by M, in bit-reversed order
    for (int k = 0; k < f.M; ++k) {
      int kb = 0;
      for (int b = 0; b < f.logM; ++b)
        if (k & (1 << b)) kb |= 1 << (f.logM - 1 - b);
      double sr = 0.0, si = 0.0;
      for (int q = 0; q < f.M; ++q) {
        double br, bi, wr, wi;
        unit_root(h.gidx[f.M + q], f.Q, br, bi);
        unit_root((int64_t)q * kb, f.M, wr, wi);
        sr += br * wr - bi * wi;
        si += br * wi + bi * wr;
      }
      t[2 * k] = sr / f.M;
      t[2 * k + 1] = si / f.M;
    }
    t += 2 * f.M;
    for (int k = 0; k < f.L; ++k, t += 2) unit_root(k, f.L, t[0], t[1]);
  }
  if (f.half)
    for (int j = 0; j <= f.N; ++j, t += 2) {
      unit_root(j, 2 * f.N, t[0], t[1]);  // exp(-i pi j / N) = (cos, -sin)
      t[1] = -t[1];
    }
  return true;
}

int fft_lines_per_cta(const FftDev& f, int elem_bytes) {
  // about 72 KB of shared memory per CTA (three CTAs per SM), at most 16 lines
  int B = 16;
  while (B > 1 && smem_of(f, B, elem_bytes) > 72 * 1024) --B;
  return B;
}

size_t fft_smem_bytes(const FftDev& f, int B, int elem_bytes) { return smem_of(f, B, elem_bytes); }

void fft_configure() {
  static bool done = false;
  if (done) return;
  cudaFuncSetAttribute(fft_axis_kernel<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFftSmemMax);
  cudaFuncSetAttribute(fft_axis_kernel<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFftSmemMax);
  cudaFuncSetAttribute(fft_axis_kernel<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFftSmemMax);
  cudaFuncSetAttribute(fft_axis_kernel<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFftSmemMax);
  done = true;
}

// axis 0: lines along x (contiguous), one per (z, y); axis 1: lines along y, one per (z, x).
template <typename T>
void launch_fft_axis(const FftDev& f, int axis, int inv, const Geom& g, const T* in, T* out, cudaStream_t s) {
  FftLines ln;
  ln.N = g.N;
  if (axis == 0) {
    ln.rows = g.my * g.mz;
    ln.rdiv = ln.rows;
    ln.hi = 0;
    ln.lo = g.mx;
    ln.es = 1;
  } else {
    ln.rows = g.mx * g.mz;
    ln.rdiv = g.mx;
    ln.hi = (int64_t)g.mx * g.my;
    ln.lo = 1;
    ln.es = g.mx;
  }
  const int B = fft_lines_per_cta(f, (int)sizeof(T));
  const size_t sm = smem_of(f, B, (int)sizeof(T));
  const unsigned grid = (unsigned)((ln.rows + B - 1) / B);
  note_launch();
  if (axis == 0)
    fft_axis_kernel<T, true><<<grid, 256, sm, s>>>(f, in, out, ln, B, inv);
  else
    fft_axis_kernel<T, false><<<grid, 256, sm, s>>>(f, in, out, ln, B, inv);
}

template void launch_fft_axis<double>(const FftDev&, int, int, const Geom&, const double*, double*, cudaStream_t);
template void launch_fft_axis<float>(const FftDev&, int, int, const Geom&, const float*, float*, cudaStream_t);

}  // namespace helm6
