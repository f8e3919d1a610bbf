// mlp_rev.cu -- (a1, reverse mode) residual network value f_D and input
// Jacobian J_D on the tensor cores by one forward pass of the values and one
// backward pass of the three output adjoints (the same f_D, J_D of Eq. 4,
// Sec. III-A; 1 + 3 columns per node and layer instead of the 18 of forward
// mode).  Split BF16 operands (hi + lo, ~16 significant bits) throughout.
//
// Per tile of NPC nodes (one CTA, persistent), with a_1 = tanh(W_0 z + b_0),
// a_{l+1} = tanh(W_l a_l + b_l) for the hidden layers and d_l = 1 - a_l^2:
//   forward:  a_1 (SIMT, FP32), a_2 .. a_{L} (MMAs with W_l), f_D = W_L a_L + b_L;
//             d_l goes to a per-CTA FP32 scratch (L2-resident)
//   backward: D_L = d_L (.) W_L'         (3 adjoint columns per node, SIMT)
//             D_l = d_l (.) (W_l' D_{l+1})  for l = L-1 .. 1   (MMAs with W_l')
//             J_D = W_0' D_1             (MMAs with W_0' as hi + lo rows)
// The activation buffer X (K = hidden width, 128 columns, N-major) holds the
// values (columns n hi, 32 + n lo) in the forward pass and the adjoints
// (columns 3n + i hi, 64 + 3n + i lo) in the backward pass; every GEMM is
// M x N x K = 128-row tiles x (64 or 128) x hidden width.  The weights of
// all GEMMs sit in one stacked BF16 tensor: W_1..W_{L-1}, W_L (rows padded to
// 128), W_1'..W_{L-1}', W_0' hi, W_0' lo (each padded to 128 rows).
//
// Roles as in mlp_tc.cu: warp 0 TMA, warp 1 tensor memory + MMA issue, warps
// 2..9 epilogue (TMEM lane quadrant = warp % 4; the two warps of a quadrant
// split the columns).  Block-granular dataflow between GEMMs (xready/xfree
// per 128-row block), bounded waits everywhere (RTN_E_TIMEOUT).
#include <algorithm>
#include <cstring>

#include "tc_common.cuh"

namespace rtn {
namespace {

constexpr int REV_CF = 32;   // forward columns per half (hi at 0, lo at 32)
constexpr int REV_CB = 64;   // backward columns per half (hi at 0, lo at 64)
constexpr int REV_CX = 128;  // columns of the activation buffer

struct RevArgs {
  const float* x;
  const float* u;
  const int* node_inst;
  int n_nodes;
  const float* W0;    // [17][HP] FP32 input layer (transposed)
  const float* b0;    // [HP]
  const float* bias;  // hidden biases [n_hidden_mm * HP] then output [>= 3]
  const float* WL;    // [3][HP] FP32 output layer
  int HP;
  int n_hidden_mm;
  uint32_t tmem_cols;
  float* fD;
  float* JD;
  float* dscr;  // [gridDim.x][n_hidden_mm + 1][NPC][HP] FP32: d_l of the tile
  int* err;
  unsigned long long* trace;
};

// GEMM g of a tile (0 <= g < 2 nh + 2): weight row base, M tiles, and kind
struct RevLayer {
  int row0;  // first weight row (of M tile 0; B0's lo rows are +128)
  int mts;   // M tiles of 128 rows
  bool bwd;  // backward: N = 128 adjoint columns, else N = 64 value columns
  bool two;  // B0: two K passes (hi rows, then lo rows)
};

__device__ __forceinline__ RevLayer rev_layer(int g, int nh, int HP) {
  const int n_mt = HP / 128, tb = nh * HP + 128;
  if (g < nh) return {g * HP, n_mt, false, false};                       // W_{g+1}
  if (g == nh) return {nh * HP, 1, false, false};                         // W_L
  if (g < 2 * nh + 1) return {tb + (2 * nh - g) * HP, n_mt, true, false};  // W_l', l = 2nh+1-g
  return {tb + nh * HP, 1, true, true};                                   // W_0' hi | lo
}

// phase trace of CTA 0 (rtn_tc_trace): entry (it * (n_gemm + 1) + g) * 8 + f
// for the it-th tile of the CTA and GEMM g; fields 0/1 MMA issue start/end
// (globaltimer ns), 2/3 epilogue start/end, 4/5/6 MMA wait cycles on
// activations / weights / accumulator slots, 7 epilogue wait cycles.  Row
// g = n_gemm holds the SIMT phases: 0/1 the last-layer adjoints, 2/3 the
// input layer.
__device__ __forceinline__ void rev_trace(const RevArgs& a, int it, int g, int n_gemm, int f,
                                          unsigned long long v) {
  const int idx = (it * (n_gemm + 1) + g) * 8 + f;
  if (idx < (1 << 16)) a.trace[idx] = v;
}

// accumulator slot of GEMM g's M tile m: single-tile GEMMs use the last slot
__device__ __forceinline__ int rev_slot(const RevLayer& L, int m, int n_mt) {
  return L.mts == 1 ? n_mt - 1 : m;
}

template <int NPC, int STAGES>
__global__ void __launch_bounds__(THREADS, 1)
    mlp_rev_kernel(const __grid_constant__ CUtensorMap tmap, RevArgs a) {
  static_assert(NPC <= REV_CF && 3 * NPC <= REV_CB, "columns");
  constexpr int NZV = NPC * NZ;
  constexpr int MT = 4;  // hidden width <= 512
  extern __shared__ uint8_t smem_raw[];
  const int HP = a.HP, nkb = HP / 64, n_mt = HP / 128;
  const int nh = a.n_hidden_mm, n_gemm = 2 * nh + 2;
  const int n_tiles = (a.n_nodes + NPC - 1) / NPC;
  const uint32_t sraw = smem_u32(smem_raw);
  const uint32_t pad = (1024u - (sraw & 1023u)) & 1023u;
  uint8_t* sm = smem_raw + pad;
  const uint32_t sbase = sraw + pad;
  const uint32_t xbytes = (uint32_t)REV_CX * HP * 2u;
  uint8_t* X = sm;
  const uint32_t x_s = sbase;
  const uint32_t w_s = sbase + xbytes;
  uint8_t* tail_area = sm + xbytes + STAGES * WT_BYTES;
  const uint32_t bar_s = smem_u32(tail_area);
  auto full_bar = [&](int s) { return bar_s + 8u * s; };
  auto empty_bar = [&](int s) { return bar_s + 8u * (STAGES + s); };
  auto acc_full = [&](int m) { return bar_s + 8u * (2 * STAGES + m); };
  auto tmem_free = [&](int m) { return bar_s + 8u * (2 * STAGES + MT + m); };
  auto xready = [&](int j) { return bar_s + 8u * (2 * STAGES + 2 * MT + j); };
  auto xfree = [&](int j) { return bar_s + 8u * (2 * STAGES + 3 * MT + j); };
  const uint32_t z_full = bar_s + 8u * (2 * STAGES + 4 * MT), z_free = z_full + 8u;
  const uint32_t fwd_done = z_full + 16u, bwd_done = z_full + 24u;
  constexpr int NBAR = 2 * STAGES + 4 * MT + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tail_area + 8 * NBAR);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* zbuf = reinterpret_cast<float*>(tail_area + 8 * NBAR + 16);
  float* dscr = a.dscr + (size_t)blockIdx.x * (nh + 1) * HP * NPC;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int m = 0; m < MT; ++m) {
      mbar_init(acc_full(m), 1);
      mbar_init(tmem_free(m), EPI_WARPS);
      mbar_init(xready(m), EPI_WARPS);
      mbar_init(xfree(m), 1);
    }
    mbar_init(z_full, EPI_WARPS);
    mbar_init(z_free, EPI_WARPS);
    mbar_init(fwd_done, EPI_WARPS);
    mbar_init(bwd_done, EPI_WARPS);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer (whole warp, one elected lane issues):
    // the weight tiles of every GEMM in order
    if (lane == 0)
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap)) : "memory");
    {
      int s = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x)
        for (int g = 0; g < n_gemm && ok; ++g) {
          const RevLayer L = rev_layer(g, nh, HP);
          const int nks = L.two ? 2 * nkb : nkb;
          for (int m = 0; m < L.mts && ok; ++m)
            for (int kb = 0; kb < nks && ok; ++kb) {
              if (!(ok = mbar_wait_warp(empty_bar(s), ph ^ 1u, abort_flag, a.err))) break;
              if (elect_one()) {
                mbar_expect_tx(full_bar(s), WT_BYTES);
                const int row = L.row0 + m * 128 + (kb >= nkb ? 128 : 0);
                const int kk = kb % nkb;
#pragma unroll
                for (int bx = 0; bx < W_BOXES; ++bx)
                  tma_load_2d(w_s + s * WT_BYTES + bx * 4096u, &tmap, kk * 64 + bx * W_BOX_K, row,
                              full_bar(s));
              }
              __syncwarp();
              if (++s == STAGES) { s = 0; ph ^= 1u; }
            }
        }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer (whole warp, one elected lane issues)
    {
      constexpr uint32_t id_f = idesc_bf16(128, 2 * REV_CF) | (1u << 16);  // B is N-major
      constexpr uint32_t id_b = idesc_bf16(128, 2 * REV_CB) | (1u << 16);
      const uint32_t lbo = REV_CX * 16u;
      int s = 0;
      uint32_t ph = 0, used = 0, tf_par = 0, xr_par = 0;
      bool ok = true;
      const bool tr = RTN_TRACE && a.trace != nullptr && blockIdx.x == 0;
      WaitClock wc(tr);
      for (int tile = blockIdx.x, it = 0; tile < n_tiles && ok; tile += gridDim.x, ++it)
        for (int g = 0; g < n_gemm && ok; ++g) {
          const RevLayer L = rev_layer(g, nh, HP);
          const int nks = L.two ? 2 * nkb : nkb;
          const uint32_t idesc = L.bwd ? id_b : id_f;
          long long w_x = 0, w_w = 0, w_t = 0;
          if (tr && lane == 0) rev_trace(a, it, g, n_gemm, 0, gtime());
          for (int m = 0; m < L.mts && ok; ++m) {
            const int slot = rev_slot(L, m, n_mt);
            if (used & (1u << slot)) {
              wc.start();
              if (!(ok = mbar_wait_warp(tmem_free(slot), (tf_par >> slot) & 1u, abort_flag, a.err))) break;
              wc.stop(w_t);
              tf_par ^= 1u << slot;
            }
            used |= 1u << slot;
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)(slot * REV_CX);
            for (int kb = 0; kb < nks && ok; ++kb) {
              const int kk = kb % nkb, j = kk >> 1;
              if (m == 0 && kb < nkb && (kk & 1) == 0) {
                wc.start();
                if (!(ok = mbar_wait_warp(xready(j), (xr_par >> j) & 1u, abort_flag, a.err))) break;
                wc.stop(w_x);
                xr_par ^= 1u << j;
                tc_fence_after();
              }
              wc.start();
              if (!(ok = mbar_wait_warp(full_bar(s), ph, abort_flag, a.err))) break;
              wc.stop(w_w);
              tc_fence_after();
              const uint32_t as = w_s + s * WT_BYTES;
#pragma unroll
              for (int ks = 0; ks < 4; ++ks) {
                const uint32_t bo = (uint32_t)(kk * 4 + ks) * 2u * lbo;  // 16 k = 2 k-groups
                mma_bf16_elect(d, wdesc(as, ks), xdesc(x_s + bo, lbo), idesc, (kb | ks) != 0);
              }
              mma_commit_elect(empty_bar(s));
              if (++s == STAGES) { s = 0; ph ^= 1u; }
              // the GEMM's last read of block j: it may be rewritten
              if (m == L.mts - 1 && kb >= nks - nkb && (kk & 1)) mma_commit_elect(xfree(j));
            }
            if (ok) mma_commit_elect(acc_full(slot));
          }
          if (tr && lane == 0) {
            rev_trace(a, it, g, n_gemm, 1, gtime());
            rev_trace(a, it, g, n_gemm, 4, w_x);
            rev_trace(a, it, g, n_gemm, 5, w_w);
            rev_trace(a, it, g, n_gemm, 6, w_t);
          }
        }
    }
  } else {
    // ---------------- epilogue warps
    const int e = warp - 2;           // 0..7
    const int q = warp & 3;           // TMEM lane quadrant
    const int half = e >> 2;          // forward: node chunk; backward: column half
    const int et = threadIdx.x - 64;  // 0..255
    for (uint32_t o = (uint32_t)et * 16u; o < xbytes; o += 256u * 16u)
      *reinterpret_cast<uint4*>(sm + o) = make_uint4(0u, 0u, 0u, 0u);
    auto ldz = [&](int node, int j) -> float {
      if (node >= a.n_nodes) return 0.0f;
      return j < NX ? a.x[(size_t)(node + a.node_inst[node]) * NX + j]
                    : a.u[(size_t)node * NU + (j - NX)];
    };
    // the tile's inputs z (NPC x 17 values, up to two per epilogue thread)
    static_assert(NZV <= 512 && NPC <= 32, "z staging");
    float zpref[2];
    auto prefetch_z = [&](int tile) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int e2 = et + 256 * h;
        zpref[h] = e2 < NZV ? ldz(tile * NPC + e2 / NZ, e2 % NZ) : 0.0f;
      }
    };
    prefetch_z(blockIdx.x);
    uint32_t acc_par = 0, xf_par = 0, zf_par = 0, zr_ph = 0, fd_par = 0, bd_par = 0;
    bool ok = true, first = true;
    const bool etr = RTN_TRACE && a.trace != nullptr && blockIdx.x == 0 && e == 0 && lane == 0;
    long long ew = 0;  // wait cycles of the current phase (traced thread)
    auto wwait = [&](uint32_t bar, uint32_t par) -> bool {
      int w_ok = 0;
      if (lane == 0) {
        const long long t0 = etr ? clock64() : 0;
        w_ok = mbar_wait(bar, par, abort_flag, a.err);
        if (etr) ew += clock64() - t0;
      }
      return __shfl_sync(0xffffffffu, w_ok, 0) != 0;
    };
    auto mark = [&](int it, int g, int f) {
      if (etr) rev_trace(a, it, g, n_gemm, f, gtime());
    };
    auto mark_end = [&](int it, int g) {
      if (etr) {
        rev_trace(a, it, g, n_gemm, 3, gtime());
        rev_trace(a, it, g, n_gemm, 7, ew);
      }
      ew = 0;
    };
    // d_l of row r: node n at dptr(l, r)[n * HP] (a warp's rows are contiguous)
    auto dptr = [&](int layer, int r) -> float* { return dscr + (size_t)layer * NPC * HP + r; };
    // 16 consecutive columns (two core-matrix groups) of row r as hi | lo
    auto put16 = [&](int r, int c_hi, int c_lo, const float* v) {
#pragma unroll
      for (int h = 0; h < 2; ++h)
        x_store8<1>(X, xoff<REV_CX>(r, c_hi + 8 * h), xoff<REV_CX>(r, c_lo + 8 * h), v + 8 * h);
    };
    auto publish = [&](int m) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(xready(m));
    };
    auto release_tmem = [&](int slot) {
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tmem_free(slot));
    };
    auto take_acc = [&](int slot) -> bool {
      if (!wwait(acc_full(slot), (acc_par >> slot) & 1u)) return false;
      acc_par ^= 1u << slot;
      tc_fence_after();
      return true;
    };
    auto take_block = [&](int m) -> bool {
      if (!wwait(xfree(m), (xf_par >> m) & 1u)) return false;
      xf_par ^= 1u << m;
      return true;
    };
    // hi + lo accumulator halves of 16 columns
    auto acc16 = [&](uint32_t taddr, int lo_off, float* v) {
      float w[16];
      tmem_ld16(taddr, v);
      tmem_ld16(taddr + lo_off, w);
      tmem_wait_ld();
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] += w[i];
    };

    // input layer (FP32): a_1 = tanh(W_0 z + b_0), d_1 to the scratch
    auto input_layer = [&](int tile) -> bool {
      const int node0 = tile * NPC;
      const int itn = (tile - (int)blockIdx.x) / (int)gridDim.x;
      ew = 0;
      mark(itn, n_gemm, 2);
      if (!wwait(z_free, zr_ph ^ 1u)) return false;  // every warp done with the last z
      zr_ph ^= 1u;
#pragma unroll
      for (int h = 0; h < 2; ++h)
        if (et + 256 * h < NZV) zbuf[((et + 256 * h) / NZ) * ZS + (et + 256 * h) % NZ] = zpref[h];
      __syncwarp();
      if (lane == 0) mbar_arrive(z_full);
      if (!wwait(z_full, zf_par)) return false;
      zf_par ^= 1u;
      // every warp has read the previous tile's d (its backward pass)
      if (!first) {
        if (!wwait(bwd_done, bd_par)) return false;
        bd_par ^= 1u;
      }
      for (int m = 0; m < n_mt; ++m) {
        if (!first && !take_block(m)) return false;
        const int r = 128 * m + 32 * q + lane;
        float w[NZ];
#pragma unroll
        for (int jj = 0; jj < NZ; ++jj) w[jj] = a.W0[(size_t)jj * HP + r];
        const float bi = a.b0[r];
        // nodes 16 half + t in batched phases
        float v[16];
#pragma unroll
        for (int g8 = 0; g8 < 2; ++g8) dot17_x8(w, zbuf, 16 * half + 8 * g8, NPC, bi, v + 8 * g8);
        tanh_batch<16>(v);
        act_finish<16>(v, dptr(0, r) + (size_t)16 * half * HP, HP, min(NPC, a.n_nodes - node0) - 16 * half,
                       NPC - 16 * half);
        put16(r, 16 * half, REV_CF + 16 * half, v);
        publish(m);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(z_free);
      first = false;
      mark_end(itn, n_gemm);
      return true;
    };

    if (blockIdx.x < n_tiles) ok = input_layer(blockIdx.x);
    for (int tile = blockIdx.x, it = 0; tile < n_tiles && ok; tile += gridDim.x, ++it) {
      const int node0 = tile * NPC;
      // forward hidden layers: a_{g+2} = tanh(W_{g+1} a_{g+1} + b)
      for (int g = 0; g < nh && ok; ++g) {
        mark(it, g, 2);
        for (int m = 0; m < n_mt; ++m) {
          const int r = 128 * m + 32 * q + lane;
          const float bi = a.bias[(size_t)g * HP + r];  // before the waits
          if (!(ok = take_acc(m))) break;
          if (!(ok = take_block(m))) break;
          const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(m * REV_CX);
          float v[16];
          acc16(trow + 16 * half, REV_CF, v);
          release_tmem(m);
          // nodes 16 half + t in batched phases
#pragma unroll
          for (int t = 0; t < 16; ++t) v[t] += bi;
          tanh_batch<16>(v);
          act_finish<16>(v, dptr(g + 1, r) + (size_t)16 * half * HP, HP,
                         min(NPC, a.n_nodes - node0) - 16 * half, NPC - 16 * half);
          put16(r, 16 * half, REV_CF + 16 * half, v);
          publish(m);
        }
        mark_end(it, g);
      }
      if (!ok) break;
      // output layer: f_D from TMEM lanes 0..2 of the last slot
      {
        const int slot = n_mt - 1;
        mark(it, nh, 2);
        if (!(ok = take_acc(slot))) break;
        if (q == 0) {
          float v[16];
          acc16(tmem + (uint32_t)(slot * REV_CX) + 16 * half, REV_CF, v);
          const float bo = lane < NO ? a.bias[(size_t)nh * HP + lane] : 0.0f;
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const int n = 16 * half + jj, node = node0 + n;
            if (n < NPC && lane < NO && node < a.n_nodes) a.fD[(size_t)node * NO + lane] = v[jj] + bo;
          }
        }
        release_tmem(slot);
        mark_end(it, nh);
      }
      // every warp has written its d of this tile
      __syncwarp();
      if (lane == 0) mbar_arrive(fwd_done);
      if (!(ok = wwait(fwd_done, fd_par))) break;
      fd_par ^= 1u;
      // adjoints of the last hidden layer: D_L = d_L (.) W_L'
      ew = 0;
      mark(it, n_gemm, 0);
      for (int m = 0; m < n_mt && ok; ++m) {
        if (!(ok = take_block(m))) break;
        const int r = 128 * m + 32 * q + lane;
        const float* dr = dptr(nh, r);
        const float wl0 = a.WL[r], wl1 = a.WL[(size_t)HP + r], wl2 = a.WL[2 * (size_t)HP + r];
#pragma unroll
        for (int c2 = 0; c2 < 2; ++c2) {
          const int c = 2 * half + c2;
          float v[16];
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const int cc = 16 * c + jj;
            const int i = cc % 3;
            v[jj] = cc < 3 * NPC ? dr[(size_t)(cc / 3) * HP] * (i == 0 ? wl0 : (i == 1 ? wl1 : wl2)) : 0.0f;
          }
          put16(r, 16 * c, REV_CB + 16 * c, v);
        }
        publish(m);
      }
      if (!ok) break;
      mark(it, n_gemm, 1);
      if (nh == 0) {
        __syncwarp();
        if (lane == 0) mbar_arrive(bwd_done);
      }
      // backward hidden layers: D_l = d_l (.) (W_l' D_{l+1}), l = nh .. 1
      for (int g = nh + 1; g <= 2 * nh && ok; ++g) {
        const int l = 2 * nh + 1 - g;
        mark(it, g, 2);
        for (int m = 0; m < n_mt; ++m) {
          if (!(ok = take_acc(m))) break;
          if (!(ok = take_block(m))) break;
          const int r = 128 * m + 32 * q + lane;
          const float* dr = dptr(l - 1, r);
          const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(m * REV_CX);
#pragma unroll
          for (int c2 = 0; c2 < 2; ++c2) {
            const int c = 2 * half + c2;
            float v[16];
            acc16(trow + 16 * c, REV_CB, v);
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) {
              const int cc = 16 * c + jj;
              v[jj] = cc < 3 * NPC ? dr[(size_t)(cc / 3) * HP] * v[jj] : 0.0f;
            }
            put16(r, 16 * c, REV_CB + 16 * c, v);
          }
          release_tmem(m);
          publish(m);
        }
        mark_end(it, g);
        if (ok && g == 2 * nh) {
          __syncwarp();
          if (lane == 0) mbar_arrive(bwd_done);
        }
      }
      if (!ok) break;
      // next tile's input layer while W_0' runs
      const int nt = tile + gridDim.x;
      if (nt < n_tiles) {
        prefetch_z(nt);
        if (!(ok = input_layer(nt))) break;
      }
      // J_D = W_0' D_1 from TMEM lanes 0..16 of the last slot
      {
        const int slot = n_mt - 1;
        mark(it, n_gemm - 1, 2);
        if (!(ok = take_acc(slot))) break;
        if (q == 0) {
          // column cc = 3 n + i is row (node0 + n) * 3 + i of J_D: entry
          // (3 node0 + cc) * 17 + lane; columns of real nodes end at `lim`
          const int lim = 3 * min(NPC, a.n_nodes - node0) - 32 * half;
          float* jrow = a.JD + ((size_t)node0 * NO + 32 * half) * NZ + lane;
#pragma unroll
          for (int c2 = 0; c2 < 2; ++c2) {
            float v[16];
            acc16(tmem + (uint32_t)(slot * REV_CX) + 16 * (2 * half + c2), REV_CB, v);
#pragma unroll
            for (int jj = 0; jj < 16; ++jj)
              if (16 * c2 + jj < lim && lane < NZ) jrow[(16 * c2 + jj) * NZ] = v[jj];
          }
        }
        release_tmem(slot);
        mark_end(it, n_gemm - 1);
      }
    }
    // tail: the last GEMM's release of every block (its commit lands here)
    if (ok && blockIdx.x < n_tiles)
      for (int m = 0; m < n_mt && ok; ++m) ok = take_block(m);
  }

  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols)
                 : "memory");
  }
}

}  // namespace

cudaError_t mlp_rev_launch(rtn_ctx* ctx, const float* x, const float* u, float* fD, float* JD) {
  TcNet& tc = ctx->net.tc;
  RevArgs a;
  a.x = x;
  a.u = u;
  a.node_inst = ctx->lay.node_inst;
  a.n_nodes = ctx->lay.n_nodes;
  a.W0 = tc.W0;
  a.b0 = tc.b0;
  a.bias = tc.bias;
  a.WL = tc.WL32;
  a.HP = tc.h_pad;
  a.n_hidden_mm = tc.n_mm;
  a.tmem_cols = (uint32_t)tc.tmem_cols;
  a.fD = fD;
  a.JD = JD;
  a.dscr = tc.dscr;
  a.err = tc.err;
  a.trace = tc.trace;
  const CUtensorMap* map = reinterpret_cast<const CUtensorMap*>(tc.tmapR_bytes);
  void* args[] = {(void*)map, (void*)&a};
  const int n_tiles = (a.n_nodes + tc.npc - 1) / tc.npc;
  dim3 grid(std::min(n_tiles, std::max(1, tc.n_sm)));  // the scratch has n_sm CTA slots
  return cudaLaunchKernel(tc.fn, grid, dim3(THREADS), args, tc.smem, ctx->stream);
}

// kernel entry of the reverse-mode shape with npc nodes and `stages` weight
// stages, or null
const void* mlp_rev_fn(int npc, int stages) {
  if (npc == 21 && stages == 6) return (const void*)&mlp_rev_kernel<21, 6>;
  if (npc == 21 && stages == 4) return (const void*)&mlp_rev_kernel<21, 4>;
  if (npc == 16 && stages == 6) return (const void*)&mlp_rev_kernel<16, 6>;
  return nullptr;
}

}  // namespace rtn
