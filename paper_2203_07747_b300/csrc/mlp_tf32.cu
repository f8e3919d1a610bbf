// mlp_tf32.cu -- the residual network's value, input Jacobian and (second
// order) Hessian at every node with FP32 accuracy on the tensor cores: the
// local models of Eq. 4 for RTN_FP32 contexts.
//
// Forward-mode differentiation carries columns per node through the network:
//   first order (MODE 1): the value and the 17 tangents t_j = da/dz_j, 18
//     columns per node, 8 nodes per tile (N = 144);
//   second order (MODE 2): also the 153 second derivatives s_jm =
//     d^2 a / dz_j dz_m (j <= m), 171 columns padded to 176, one node per
//     tile (N = 176).
// A hidden neuron with pre-activation columns (z_0, z_j, z_jm) produces
//   a = tanh(z_0 + b),  t_j = tanh'(.) z_j,  s_jm = tanh'(.) z_jm + tanh''(.) z_j z_m,
// with tanh' = 1 - a^2, tanh'' = -2 a (1 - a^2).
//
// Layout: activations are stored transposed, X' [node * CPN + column][hs]
// (CPN = 18 or 176 columns per node), as TF32 hi + lo pairs (v = hi + lo to
// about 2^-22), so that a hidden->hidden layer Z = W X is one tensor-core GEMM
// per (128-neuron tile, node group): M = 128 neurons, N = the group's columns,
// K = the layer's input width, both operands K-major, three kind::tf32 MMAs
// per K step (hi hi + hi lo + lo hi, FP32 accumulation in TMEM).  A TMEM lane
// then holds every column of one neuron for the nodes of the tile, so the
// activation rule above is thread-local and runs in the GEMM's epilogue,
// which writes the next layer's X' directly (tf_tc_kernel).  The input layer
// (no GEMM: its tangents are W_0's columns and its second derivatives the
// rank-one d2 w_j w_m) and the 3- or 6-row output layer run on the SIMT
// cores (tf_in_kernel, tf_out_kernel).
#include <algorithm>
#include <cstring>
#include <new>
#include <utility>

#include "tc_common.cuh"

namespace rtn {
namespace {

constexpr int C2 = 1 + NZ + NZ * (NZ + 1) / 2;  // 171 second-order columns per node
constexpr int TF_KB = 32;                       // K per stage: one 128 B swizzle row of FP32
constexpr uint32_t TF_A_BYTES = 128u * TF_KB * 4u;  // weight tile, 16 KB
constexpr int TF_THREADS = 192;                 // warp 0 TMA, warp 1 MMA, warps 2..5 epilogue
constexpr uint32_t TF_TMEM_COLS = 512;          // two accumulators, 256 columns apart
constexpr int TF_NBAR_MAX = 2 * 3 + 5;

// shape of a mode: columns per node (padded), columns used, nodes per tile,
// the MMA's N, pipeline stages
template <int MODE>
struct Tf;
template <>
struct Tf<1> {
  static constexpr int CPN = NC, CUSED = NC, NPT = 8, N = NC * 8, STAGES = 3;
};
template <>
struct Tf<2> {
  static constexpr int CPN = 176, CUSED = C2, NPT = 1, N = 176, STAGES = 2;
};

template <int MODE>
__host__ __device__ constexpr uint32_t tf_b_bytes() { return (uint32_t)Tf<MODE>::N * TF_KB * 4u; }
template <int MODE>
__host__ __device__ constexpr uint32_t tf_stage() { return 2u * TF_A_BYTES + 2u * tf_b_bytes<MODE>(); }
template <int MODE>
__host__ __device__ constexpr size_t tf_smem() { return Tf<MODE>::STAGES * tf_stage<MODE>() + 1024 + 256; }

static_assert(tf_b_bytes<1>() % 1024 == 0 && tf_b_bytes<2>() % 1024 == 0, "swizzled tiles stay 1 KB aligned");
static_assert(Tf<1>::N % 16 == 0 && Tf<2>::N % 16 == 0 && Tf<2>::N <= 256, "MMA N");
static_assert(tf_smem<1>() <= 232448 && tf_smem<2>() <= 232448, "shared memory");

// pair (j, m), j <= m, of second-derivative column 18 + p (row-major upper
// triangle)
__host__ __device__ constexpr int pair_j(int p) {
  int j = 0;
  while (p >= NZ - j) { p -= NZ - j; ++j; }
  return j;
}
__host__ __device__ constexpr int pair_m(int p) {
  int j = 0;
  while (p >= NZ - j) { p -= NZ - j; ++j; }
  return j + p;
}

__constant__ unsigned char k_pj[NZ * (NZ + 1) / 2];
__constant__ unsigned char k_pm[NZ * (NZ + 1) / 2];

struct TfMaps {
  CUtensorMap wh, wl, xh, xl;
};

// round to TF32 (10 explicit mantissa bits), nearest, ties away from zero
__device__ __forceinline__ float tf32_rna(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}

__device__ __forceinline__ void split_store(float* __restrict__ hi, float* __restrict__ lo, size_t idx, float v) {
  const float h = tf32_rna(v);
  hi[idx] = h;
  lo[idx] = tf32_rna(v - h);
}

// instruction descriptor, kind::tf32: D f32, A = B = tf32, both K-major
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32_elect(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                               uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p, e;\n\tsetp.ne.b32 p, %4, 0;\n\telect.sync _|e, 0xffffffff;\n\t"
      "@e tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}

// ---------------------------------------------------------------- input layer
// thread (neuron i, node n): pre-activation s = b_i + w_i . z_n, then every
// column of the node: a, d1 w_ij (and d2 w_ij w_im, zero padding)
template <int MODE>
__global__ void __launch_bounds__(256) tf_in_kernel(const float* __restrict__ x, const float* __restrict__ u,
                                                    const int* __restrict__ node_inst, int n_nodes,
                                                    const float* __restrict__ W0, const float* __restrict__ b0,
                                                    int h1, int hs, float* __restrict__ xh, float* __restrict__ xl) {
  constexpr int CPN = Tf<MODE>::CPN;
  const int i = blockIdx.x * 32 + threadIdx.x;
  const bool act = i < h1;
  const float* w = W0 + (size_t)(act ? i : 0) * NZ;
  for (int n = blockIdx.y * 8 + threadIdx.y; n < n_nodes; n += gridDim.y * 8) {
    const float* xr = x + (size_t)(n + node_inst[n]) * NX;
    const float* ur = u + (size_t)n * NU;
    float s = b0[act ? i : 0];
#pragma unroll
    for (int j = 0; j < NX; ++j) s = fmaf(__ldg(w + j), xr[j], s);
#pragma unroll
    for (int j = 0; j < NU; ++j) s = fmaf(__ldg(w + NX + j), ur[j], s);
    const float a = tanhf(s), d1 = 1.0f - a * a, d2 = -2.0f * a * d1;
    if (!act) continue;
    const size_t row0 = (size_t)n * CPN;
    for (int c = 0; c < CPN; ++c) {
      float v;
      if (c == 0) v = a;
      else if (c <= NZ) v = d1 * __ldg(w + c - 1);
      else if (c < C2) v = d2 * __ldg(w + k_pj[c - 1 - NZ]) * __ldg(w + k_pm[c - 1 - NZ]);
      else v = 0.0f;
      split_store(xh, xl, (row0 + c) * hs + i, v);
    }
  }
}

// --------------------------------------------------------------- output layer
// one warp per (node n, column c): out_r = WL_r . (xh + xl)[row], the lanes
// splitting K; writes f_D [n][NOUT], J_D [n][NOUT][17] and (MODE 2) H_D
// [n][NOUT][17][17] (both triangles)
template <int MODE, int NOUT>
__global__ void __launch_bounds__(256) tf_out_kernel(const float* __restrict__ WL, const float* __restrict__ bL,
                                                     int h, int n_nodes, int hs, const float* __restrict__ xh,
                                                     const float* __restrict__ xl, float* __restrict__ fD,
                                                     float* __restrict__ JD, float* __restrict__ HD) {
  constexpr int CPN = Tf<MODE>::CPN, CU = Tf<MODE>::CUSED;
  const int lane = threadIdx.x & 31;
  const long long total = (long long)n_nodes * CU;
  for (long long wq = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; wq < total;
       wq += ((long long)gridDim.x * blockDim.x) >> 5) {
    const int n = (int)(wq / CU), c = (int)(wq % CU);
    const size_t row = ((size_t)n * CPN + c) * hs;
    float acc[NOUT];
#pragma unroll
    for (int r = 0; r < NOUT; ++r) acc[r] = 0.0f;
    for (int k = lane; k < h; k += 32) {
      const float xv = __ldg(xh + row + k) + __ldg(xl + row + k);
#pragma unroll
      for (int r = 0; r < NOUT; ++r) acc[r] = fmaf(__ldg(WL + (size_t)r * h + k), xv, acc[r]);
    }
#pragma unroll
    for (int r = 0; r < NOUT; ++r)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
    if (lane != 0) continue;
#pragma unroll
    for (int r = 0; r < NOUT; ++r) {
      if (c == 0) {
        fD[(size_t)n * NOUT + r] = acc[r] + bL[r];
      } else if (c <= NZ) {
        JD[((size_t)n * NOUT + r) * NZ + (c - 1)] = acc[r];
      } else if (MODE == 2) {
        const int p = c - 1 - NZ, j = k_pj[p], m = k_pm[p];
        float* Hr = HD + ((size_t)n * NOUT + r) * NZ * NZ;
        Hr[j * NZ + m] = acc[r];
        Hr[m * NZ + j] = acc[r];
      }
    }
  }
}

// ------------------------------------------------- hidden layers (tcgen05)

struct EpiOut {
  float* yh;
  float* yl;
  size_t row0;  // first row of the tile in X'
  int hs, i;
  bool active;  // neuron i exists
  int n_valid;  // nodes of the tile that exist
  float bias;
};

// MODE 2: the activated value of column C from its pre-activation z (C is a
// compile-time constant, so the pair (j, m) of a second-derivative column
// indexes the tangent registers statically)
template <int C>
__device__ __forceinline__ float h2_val(float z, float a, float d1, float d2, const float (&t)[NZ]) {
  if constexpr (C == 0) {
    return a;
  } else if constexpr (C <= NZ) {
    return d1 * z;
  } else if constexpr (C < C2) {
    constexpr int J = pair_j(C - 1 - NZ), M = pair_m(C - 1 - NZ);
    return fmaf(d2, t[J] * t[M], d1 * z);
  } else {
    return 0.0f;
  }
}

template <int K, int... Q>
__device__ __forceinline__ void h2_emit(const float (&v)[16], float a, float d1, float d2, const float (&t)[NZ],
                                        const EpiOut& o, std::integer_sequence<int, Q...>) {
  if (o.active)
    (split_store(o.yh, o.yl, (o.row0 + 16 * K + Q) * o.hs + o.i, h2_val<16 * K + Q>(v[Q], a, d1, d2, t)), ...);
}

// chunks K .. 10 of 16 columns: load from TMEM, activate, store
template <int K>
__device__ __forceinline__ void h2_rest(uint32_t taddr, float a, float d1, float d2, const float (&t)[NZ],
                                        const EpiOut& o) {
  if constexpr (K < Tf<2>::N / 16) {
    float v[16];
    tmem_ld16(taddr + 16 * K, v);
    tmem_wait_ld();
    h2_emit<K>(v, a, d1, d2, t, o, std::make_integer_sequence<int, 16>{});
    h2_rest<K + 1>(taddr, a, d1, d2, t, o);
  }
}

// MODE 1: column C of the tile is column C % 18 of its node C / 18; the
// node's value column comes first and sets a, tanh' for its tangents
template <int C>
__device__ __forceinline__ void f1_col(float z, float& a, float& d1, const EpiOut& o) {
  constexpr int k = C / NC, c = C % NC;
  float v;
  if constexpr (c == 0) {
    a = tanhf(z + o.bias);
    d1 = 1.0f - a * a;
    v = a;
  } else {
    v = d1 * z;
  }
  if (o.active && k < o.n_valid) split_store(o.yh, o.yl, (o.row0 + C) * o.hs + o.i, v);
}

template <int K, int... Q>
__device__ __forceinline__ void f1_emit(const float (&v)[16], float& a, float& d1, const EpiOut& o,
                                        std::integer_sequence<int, Q...>) {
  (f1_col<16 * K + Q>(v[Q], a, d1, o), ...);
}

template <int K>
__device__ __forceinline__ void f1_rest(uint32_t taddr, float& a, float& d1, const EpiOut& o) {
  if constexpr (K < Tf<1>::N / 16) {
    float v[16];
    tmem_ld16(taddr + 16 * K, v);
    tmem_wait_ld();
    f1_emit<K>(v, a, d1, o, std::make_integer_sequence<int, 16>{});
    f1_rest<K + 1>(taddr, a, d1, o);
  }
}

// One hidden->hidden layer: tiles (node group, neuron tile mt) in group-major
// order over persistent CTAs (the MT tiles of a group read its X' block while
// it is in L2); K in stages of 32; two TMEM accumulators so that the epilogue
// of one tile overlaps the MMAs of the next.
template <int MODE>
__global__ void __launch_bounds__(TF_THREADS, 1)
    tf_tc_kernel(const __grid_constant__ TfMaps maps, const float* __restrict__ bias, int ho, int kp, int n_nodes,
                 int hs, float* __restrict__ yh, float* __restrict__ yl, int* err) {
  using T = Tf<MODE>;
  constexpr int S_N = T::STAGES;
  constexpr uint32_t B_BYTES = tf_b_bytes<MODE>(), STAGE = tf_stage<MODE>();
  extern __shared__ uint8_t smem_raw[];
  const uint32_t sraw = smem_u32(smem_raw);
  const uint32_t pad = (1024u - (sraw & 1023u)) & 1023u;
  uint8_t* sm = smem_raw + pad;
  const uint32_t st0 = sraw + pad;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + S_N * STAGE);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + TF_NBAR_MAX);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  auto bar = [&](int k) { return smem_u32(bars + k); };
  auto full_bar = [&](int s) { return bar(s); };
  auto empty_bar = [&](int s) { return bar(S_N + s); };
  auto acc_full = [&](int a) { return bar(2 * S_N + a); };
  auto tmem_free = [&](int a) { return bar(2 * S_N + 2 + a); };
  const uint32_t mma_done = bar(2 * S_N + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int MT = (ho + 127) / 128;
  const int n_groups = (n_nodes + T::NPT - 1) / T::NPT;
  const long long n_tiles = (long long)n_groups * MT;
  const int nkb = kp / TF_KB;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S_N; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(acc_full(a), 1);
      mbar_init(tmem_free(a), 4);
    }
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TF_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.wh)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.xh)) : "memory");
    }
    int s = 0;
    uint32_t ph = 0;
    bool ok = true;
    uint32_t issued = 0, last_ph = 0;  // per stage: a load was issued / its phase parity
    for (long long t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
      const int grp = (int)(t / MT), mt = (int)(t % MT);
      for (int kb = 0; kb < nkb; ++kb) {
        if (!(ok = mbar_wait_warp(empty_bar(s), ph ^ 1u, abort_flag, err))) break;
        if (elect_one()) {
          const uint32_t sa = st0 + s * STAGE;
          mbar_expect_tx(full_bar(s), STAGE);
          tma_load_2d(sa, &maps.wh, kb * TF_KB, mt * 128, full_bar(s));
          tma_load_2d(sa + TF_A_BYTES, &maps.wl, kb * TF_KB, mt * 128, full_bar(s));
          tma_load_2d(sa + 2 * TF_A_BYTES, &maps.xh, kb * TF_KB, grp * T::N, full_bar(s));
          tma_load_2d(sa + 2 * TF_A_BYTES + B_BYTES, &maps.xl, kb * TF_KB, grp * T::N, full_bar(s));
        }
        __syncwarp();
        issued |= 1u << s;
        last_ph = (last_ph & ~(1u << s)) | (ph << s);
        if (++s == S_N) { s = 0; ph ^= 1u; }
      }
    }
    // every issued copy has landed before the CTA exits (bounded)
    for (int q = 0; q < S_N; ++q)
      if (issued & (1u << q)) {
        const long long t0 = clock64();
        while (!mbar_try(full_bar(q), (last_ph >> q) & 1u) && clock64() - t0 < WAIT_CYCLES) {
        }
      }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    constexpr uint32_t idesc = idesc_tf32(128, T::N);
    int s = 0, acc = 0;
    uint32_t ph = 0, aph = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
      if (!(ok = mbar_wait_warp(tmem_free(acc), aph ^ 1u, abort_flag, err))) break;
      tc_fence_after();
      const uint32_t d = tmem + acc * 256u;
      for (int kb = 0; kb < nkb; ++kb) {
        if (!(ok = mbar_wait_warp(full_bar(s), ph, abort_flag, err))) break;
        tc_fence_after();
        const uint32_t sa = st0 + s * STAGE;
#pragma unroll
        for (int ks = 0; ks < TF_KB / 8; ++ks) {
          const uint64_t ah = kmajor_desc(sa + ks * 32u, 1024, 2);
          const uint64_t al = kmajor_desc(sa + TF_A_BYTES + ks * 32u, 1024, 2);
          const uint64_t bh = kmajor_desc(sa + 2 * TF_A_BYTES + ks * 32u, 1024, 2);
          const uint64_t bl = kmajor_desc(sa + 2 * TF_A_BYTES + B_BYTES + ks * 32u, 1024, 2);
          mma_tf32_elect(d, ah, bh, idesc, (kb | ks) != 0);
          mma_tf32_elect(d, ah, bl, idesc, 1u);
          mma_tf32_elect(d, al, bh, idesc, 1u);
        }
        mma_commit_elect(empty_bar(s));
        if (++s == S_N) { s = 0; ph ^= 1u; }
      }
      if (!ok) break;
      mma_commit_elect(acc_full(acc));
      if (++acc == 2) { acc = 0; aph ^= 1u; }
    }
    // the MMAs issued so far have completed before TMEM is released (bounded)
    mma_commit_elect(mma_done);
    const long long t0 = clock64();
    while (!mbar_try(mma_done, 0) && clock64() - t0 < WAIT_CYCLES) {
    }
  } else {
    // ---------------- epilogue: TMEM lane quarter warp % 4
    const int q = warp & 3;
    int acc = 0;
    uint32_t aph = 0;
    for (long long t = blockIdx.x; t < n_tiles; t += gridDim.x) {
      const int grp = (int)(t / MT), mt = (int)(t % MT);
      if (!mbar_wait_warp(acc_full(acc), aph, abort_flag, err)) break;
      tc_fence_after();
      EpiOut o;
      o.yh = yh;
      o.yl = yl;
      o.row0 = (size_t)grp * T::N;
      o.hs = hs;
      o.i = mt * 128 + q * 32 + lane;
      o.active = o.i < ho;
      o.n_valid = min(T::NPT, n_nodes - grp * T::NPT);
      o.bias = o.active ? __ldg(bias + o.i) : 0.0f;
      const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + acc * 256u;
      if constexpr (MODE == 1) {
        float a = 0.0f, d1 = 0.0f;
        f1_rest<0>(taddr, a, d1, o);
      } else {
        float v0[16], v1[16];
        tmem_ld16(taddr, v0);
        tmem_ld16(taddr + 16, v1);
        tmem_wait_ld();
        const float a = tanhf(v0[0] + o.bias);
        const float d1 = 1.0f - a * a, d2 = -2.0f * a * d1;
        float tz[NZ];
#pragma unroll
        for (int j = 0; j < NZ; ++j) tz[j] = j < 15 ? v0[1 + j] : v1[j - 15];
        h2_emit<0>(v0, a, d1, d2, tz, o, std::make_integer_sequence<int, 16>{});
        h2_emit<1>(v1, a, d1, d2, tz, o, std::make_integer_sequence<int, 16>{});
        h2_rest<2>(taddr, a, d1, d2, tz, o);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tmem_free(acc));
      if (++acc == 2) { acc = 0; aph ^= 1u; }
    }
  }

  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TF_TMEM_COLS)
                 : "memory");
  }
}

// FP32 -> TF32 with round-to-nearest-even on the 13 dropped mantissa bits
float tf32_round(float v) {
  uint32_t u;
  std::memcpy(&u, &v, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) {
    u += 0x0fffu + ((u >> 13) & 1u);
    u &= 0xffffe000u;
  }
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

template <int MODE>
void tf_launch(rtn_ctx* ctx, const float* x, const float* u, float* fD, float* JD, float* HD) {
  using T = Tf<MODE>;
  Net& net = ctx->net;
  TfState* h = ctx->tf;
  const int n = ctx->lay.n_nodes, L = net.n_layers;
  cudaStream_t s = ctx->stream;
  const int h1 = net.widths[1];
  {
    dim3 grid((unsigned)((h1 + 31) / 32), (unsigned)std::min((n + 7) / 8, 65535));
    tf_in_kernel<MODE><<<grid, dim3(32, 8), 0, s>>>(x, u, ctx->lay.node_inst, n, net.W32 + net.w_off[0],
                                                   net.b32 + net.b_off[0], h1, h->hs, h->x[0][0], h->x[0][1]);
  }
  for (int l = 1; l + 1 < L; ++l) {
    const int ho = net.widths[l + 1];
    const int dst = l & 1;
    const long long tiles = (long long)((n + T::NPT - 1) / T::NPT) * ((ho + 127) / 128);
    const int grid = (int)std::min<long long>(tiles, 148);
    const TfMaps* maps = reinterpret_cast<const TfMaps*>(h->maps[l - 1].data());
    tf_tc_kernel<MODE><<<grid, TF_THREADS, tf_smem<MODE>(), s>>>(*maps, net.b32 + net.b_off[l], ho, h->kp[l - 1], n,
                                                                h->hs, h->x[dst][0], h->x[dst][1], net.tc.err);
  }
  const int last = (L - 2) & 1;  // buffer the output layer reads
  const long long warps = (long long)n * T::CUSED;
  const int grid = (int)std::min<long long>((warps + 7) / 8, 148LL * 64);
  auto out = net.widths[L] == NO_FULL ? tf_out_kernel<MODE, NO_FULL> : tf_out_kernel<MODE, NO>;
  out<<<grid, 256, 0, s>>>(net.W32 + net.w_off[L - 1], net.b32 + net.b_off[L - 1], net.widths[L - 1], n, h->hs,
                           h->x[last][0], h->x[last][1], fD, JD, HD);
}

}  // namespace

cudaError_t mlp_tf32_prepare(rtn_ctx* ctx, int mode, std::string& err) {
  unsigned char pj[NZ * (NZ + 1) / 2], pm[NZ * (NZ + 1) / 2];
  for (int p = 0; p < NZ * (NZ + 1) / 2; ++p) {
    pj[p] = (unsigned char)pair_j(p);
    pm[p] = (unsigned char)pair_m(p);
  }
  cudaError_t e = cudaMemcpyToSymbol(k_pj, pj, sizeof(pj));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(k_pm, pm, sizeof(pm));
  if (e != cudaSuccess) return e;

  Net& net = ctx->net;
  const int L = net.n_layers, n = ctx->lay.n_nodes;
  const int cpn = mode == 2 ? Tf<2>::CPN : Tf<1>::CPN;
  const int nrows_tile = mode == 2 ? Tf<2>::N : Tf<1>::N;
  const long long rows = (long long)n * cpn;
  if (rows + nrows_tile >= (1LL << 31)) {
    err = "FP32 network: more nodes than the 32-bit tensor coordinates address";
    return cudaSuccess;
  }
  TfState* h = new (std::nothrow) TfState();
  if (!h) return cudaErrorMemoryAllocation;
  ctx->tf = h;
  h->mode = mode;
  int hmax = 0;
  for (int l = 1; l < L; ++l) hmax = std::max(hmax, net.widths[l]);
  h->hs = (hmax + 31) / 32 * 32;
  const size_t xfl = (size_t)rows * h->hs;
  for (int b = 0; b < 2; ++b)
    for (int p = 0; p < 2; ++p) {
      if ((e = cudaMalloc(&h->x[b][p], xfl * sizeof(float))) != cudaSuccess) return e;
      // K entries a narrower layer never writes stay finite (zero): the
      // zero weight padding then removes them from the next GEMM
      if ((e = cudaMemset(h->x[b][p], 0, xfl * sizeof(float))) != cudaSuccess) return e;
    }
  TcNet& tc = net.tc;
  if (!tc.err) {
    if ((e = cudaMalloc(&tc.err, sizeof(int))) != cudaSuccess) return e;
    if ((e = cudaMemset(tc.err, 0, sizeof(int))) != cudaSuccess) return e;
  }
  if (L < 3) return cudaSuccess;  // one hidden layer: no GEMM

  void* fn = nullptr;
  cudaDriverEntryPointQueryResult qr;
  e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr);
  if (e != cudaSuccess || !fn || qr != cudaDriverEntryPointSuccess) {
    err = "cuTensorMapEncodeTiled unavailable";
    return cudaSuccess;
  }
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  e = mode == 2 ? cudaFuncSetAttribute(tf_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tf_smem<2>())
                : cudaFuncSetAttribute(tf_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tf_smem<1>());
  if (e != cudaSuccess) return e;
  for (int l = 1; l + 1 < L; ++l) {
    const int hi = net.widths[l], ho = net.widths[l + 1];
    const int kp = (hi + 31) / 32 * 32, wrows = (ho + 127) / 128 * 128;
    // split weights, zero padded to [wrows][kp]
    std::vector<float> W((size_t)ho * hi);
    if ((e = cudaMemcpy(W.data(), net.W32 + net.w_off[l], W.size() * 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
      return e;
    std::vector<float> wh((size_t)wrows * kp, 0.0f), wl((size_t)wrows * kp, 0.0f);
    for (int r = 0; r < ho; ++r)
      for (int k = 0; k < hi; ++k) {
        const float v = W[(size_t)r * hi + k], vh = tf32_round(v);
        wh[(size_t)r * kp + k] = vh;
        wl[(size_t)r * kp + k] = tf32_round(v - vh);
      }
    float *dh = nullptr, *dl = nullptr;
    if ((e = cudaMalloc(&dh, wh.size() * 4)) != cudaSuccess) return e;
    h->wh.push_back(dh);
    if ((e = cudaMalloc(&dl, wl.size() * 4)) != cudaSuccess) return e;
    h->wl.push_back(dl);
    if ((e = cudaMemcpy(dh, wh.data(), wh.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(dl, wl.data(), wl.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    h->kp.push_back(kp);
    // tensor maps: W hi/lo [wrows][kp], box 32 x 128; X' hi/lo of the buffer
    // this layer reads, [n * CPN][hs], box 32 x N (the last node group's box
    // may reach past the last row: those rows load as zeros and their
    // results are not stored); 128 B swizzle
    std::vector<unsigned char> m(sizeof(TfMaps));
    TfMaps* mp = reinterpret_cast<TfMaps*>(m.data());
    const cuuint32_t estr[2] = {1, 1};
    const cuuint64_t wdims[2] = {(cuuint64_t)kp, (cuuint64_t)wrows};
    const cuuint64_t wstr[1] = {(cuuint64_t)kp * 4};
    const cuuint32_t wbox[2] = {(cuuint32_t)TF_KB, 128};
    const cuuint64_t xdims[2] = {(cuuint64_t)h->hs, (cuuint64_t)rows};
    const cuuint64_t xstr[1] = {(cuuint64_t)h->hs * 4};
    const cuuint32_t xbox[2] = {(cuuint32_t)TF_KB, (cuuint32_t)nrows_tile};
    const int src = (l - 1) & 1;
    struct Enc {
      CUtensorMap* map;
      void* ptr;
      const cuuint64_t* dims;
      const cuuint64_t* str;
      const cuuint32_t* box;
    } enc[4] = {{&mp->wh, dh, wdims, wstr, wbox},
                {&mp->wl, dl, wdims, wstr, wbox},
                {&mp->xh, h->x[src][0], xdims, xstr, xbox},
                {&mp->xl, h->x[src][1], xdims, xstr, xbox}};
    for (auto& q : enc) {
      CUresult r = encode(q.map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, q.ptr, q.dims, q.str, q.box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) {
        err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
        return cudaSuccess;
      }
    }
    h->maps.push_back(std::move(m));
  }
  return cudaSuccess;
}

void mlp_tf32_release(rtn_ctx* ctx) {
  TfState* h = ctx->tf;
  if (!h) return;
  for (int b = 0; b < 2; ++b)
    for (int p = 0; p < 2; ++p)
      if (h->x[b][p]) cudaFree(h->x[b][p]);
  for (float* p : h->wh) cudaFree(p);
  for (float* p : h->wl) cudaFree(p);
  delete h;
  ctx->tf = nullptr;
}

cudaError_t mlp_tf32_forward(rtn_ctx* ctx, const float* x, const float* u, float* fD, float* JD, float* HD) {
  if (!ctx->tf) return cudaErrorInvalidValue;
  if (ctx->tf->mode == 2) {
    if (!HD) return cudaErrorInvalidValue;
    tf_launch<2>(ctx, x, u, fD, JD, HD);
  } else {
    tf_launch<1>(ctx, x, u, fD, JD, nullptr);
  }
  return cudaGetLastError();
}

}  // namespace rtn
