// Cluster-resident hierarchical and spin-2 samplers for 256 x 256 and 512 x 512 images (the two
// extensions of §5 on the cluster geometry of wf_cluster.cuh: one chain per thread-block cluster, CTA b
// keeping the global rows y = P a + b for all sweeps).
//
// Hierarchical (power spectrum inference): the s-draw takes its coefficients from the band powers held
// in every CTA's shared memory (as the per-band table band_coef(P_b)) and stores each new mode's
// statistics (n |s_hat|^2 with its mirror weight, the squares of its stream-6 normals) at the mode's own
// position of a bin-ordered buffer in global memory (one per cluster, L2-resident). After the sweep's
// second cluster barrier CTA j sums its range of bins from that buffer (a warp per bin, lane-strided
// partial sums then a fixed shuffle tree: the same order every run), draws P_b = S_b / X_b and writes
// P_b and band_coef(P_b) into the shared memory of every CTA of the cluster (and P_b to out_P when the
// sweep is kept). Those writes land before the next sweep's first barrier, and nobody reads the tables
// between the second barrier and the next first one, so no further barrier is needed; the buffer is
// rewritten only after the next first barrier, when every CTA has finished reading it.
//
// Spin-2 (shear): both shear components of a chain in one cluster, each CTA holding its rows of both
// (2 x N/2 threads, one component's row and column passes per half), and a column unit gathering the
// column spectra of both components so that the Kaiser-Squires rotation into E and B, the two scalar
// s-draws and the rotation back happen on complete mode pairs (the two units of a pair on partner lanes).
#pragma once

#include "wf_cluster.cuh"

namespace wf {

// ---------------------------------------------------------------------------------------------
// hierarchical sampler
// ---------------------------------------------------------------------------------------------
// shared bytes: rows, twiddles, per-band s-draw coefficients [n_bins] (float2), band powers [n_bins]
template <int N, int MR>
__host__ __device__ constexpr int cband_smem(int n_bins) {
  return CGeo<N, MR>::ROWS_BYTES + N * 8 + ((12 * n_bins + 15) / 16) * 16;
}

// a.band_clusters clusters; cluster c runs chains c, c + band_clusters, ... (one statistics buffer each);
// a.fg and a.band_map in slot order (ctab_index), a.aq with the CTA-contiguous rows
template <int N, int MR>
__global__ void __launch_bounds__(N / 2, csample_min_ctas<N, MR>()) k_csample_band(SampleArgs a) {
  using G = CGeo<N, MR>;
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* rows = reinterpret_cast<float2*>(smem_raw);
  float2* tw = reinterpret_cast<float2*>(smem_raw + G::ROWS_BYTES);
  float2* cb = reinterpret_cast<float2*>(smem_raw + G::ROWS_BYTES + N * 8);
  float* Pb = reinterpret_cast<float*>(cb + a.n_bins);
  if (a.sc->status != 0) return;  // uniform over the grid
  const int nb = a.n_bins, tid = threadIdx.x, b = int(cl.block_rank()), g = b * G::L + tid;
  const int cid = blockIdx.x / G::P;
  const float tau = float(a.sc->tau);
  constexpr float NPIX = float(G::H * G::W);
  float2* buf = a.band_buf + (long long)cid * (nb > 0 ? a.band_off[nb] : 0);
  const int lo = a.band_lo[b], hi = a.band_lo[b + 1];
  const int warp = tid / 32, lane = tid % 32;
  ctw_init<N, MR>(tw);
  for (long long ci = cid; ci < a.n_chains; ci += a.band_clusters) {
    for (int i = tid; i < nb; i += G::L) {
      Pb[i] = a.P0[i];
      cb[i] = band_coef(a.P0[i], tau, 1.0f / NPIX);
    }
    crows_load<N, MR>(rows, b, a.init_s ? a.init_s + ci * a.init_stride : nullptr);
    __syncthreads();
    const uint32_t chain = a.chain0 + uint32_t(ci);
    float* out_P = a.out_P ? a.out_P + ci * a.n_samples * nb : nullptr;
    const long long out_off = ci * a.n_samples * (long long)(G::H * G::W) * out_elem_bytes(a.out_dtype);
    csweeps<N, MR, 1, false>(
        cl, rows, tw, a.aq, a.sc->sqrt_tau, reinterpret_cast<char*>(a.out) + out_off, a.out_dtype, a.n_sweeps,
        a.burn_in, a.thin, a.step0, chain, a.key0, a.key1,
        [&](uint32_t step, int) {  // s-draw with P_k = P_b(k); each mode's statistics to the buffer
          ccol_draw<N, MR>(cl, rows, g, CBandCoef{a.fg, a.band_map, cb, buf, NPIX}, step, chain, a.key0, a.key1);
        },
        [&](uint32_t, int done) {  // P_b | s for this CTA's bins, to every CTA of the cluster
          const int kept = done + 1 - a.burn_in;
          const long long m = (kept > 0 && kept % a.thin == 0) ? kept / a.thin - 1 : -1;
          for (int bb = lo + warp; bb < hi; bb += G::L / 32) {
            const int o1 = a.band_off[bb + 1];
            float S = 0.0f, X = 0.0f;
            for (int j = a.band_off[bb] + lane; j < o1; j += 8 * 32) {  // eight loads in flight per lane
              float2 v[8];
#pragma unroll
              for (int u = 0; u < 8; ++u)
                v[u] = j + 32 * u < o1 ? __ldcg(buf + j + 32 * u) : make_float2(0.0f, 0.0f);
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                S += v[u].x;
                X += v[u].y;
              }
            }
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
              S += __shfl_xor_sync(0xffffffffu, S, d);
              X += __shfl_xor_sync(0xffffffffu, X, d);
            }
            const float P = X > 0.0f ? S / X : 0.0f;
            if (lane < G::P) {
              cl.map_shared_rank(Pb, lane)[bb] = P;
              cl.map_shared_rank(cb, lane)[bb] = band_coef(P, tau, 1.0f / NPIX);
            }
            if (lane == 0 && out_P && m >= 0) out_P[m * nb + bb] = P;
          }
        });
    cl.sync();  // the chain's last remote writes and reads are done before the next chain starts
  }
}

// ---------------------------------------------------------------------------------------------
// spin-2 sampler
// ---------------------------------------------------------------------------------------------
// shared bytes: the rows of both components, twiddles
template <int N, int MR>
__host__ __device__ constexpr int cspin2_smem() { return 2 * CGeo<N, MR>::ROWS_BYTES + N * 8; }
// threads per CTA: 2 L, one component's row and column passes per half (256^2: 8-CTA clusters of 256
// threads, 2 CTAs per SM; 512^2: 16-CTA clusters of 512 threads, 1 per SM), the column stage then taking
// one or two units of a pair per thread (ccol_units2)
template <int N, int MR>
__host__ __device__ constexpr bool cspin2_split() { return true; }
template <int N, int MR>
__host__ __device__ constexpr int cspin2_threads() { return cspin2_split<N, MR>() ? 2 * CGeo<N, MR>::L : CGeo<N, MR>::L; }
template <int N, int MR>
__host__ __device__ constexpr int cspin2_min_ctas() { return 2 * (cspin2_smem<N, MR>() + 1024) <= 228 * 1024 ? 2 : 1; }

// The spin-2 s-draw of one mode pair (ky1, ky2) of packed column slot t (kx = K) on both components
// (y1a, y2a: component 1; y1b, y2b: component 2): per mode, rotation by (c, s) = (cos 2 phi, sin 2 phi)
// into E and B, the scalar draws with tables fgE, fgB (slot order, (f / n, g / sqrt(2 n)) of P_E, P_B;
// zeta_E from stream 1, zeta_B from stream 9, in the scalar draw's counter layout), rotation back. The
// packed edge column is unpacked into (ky1, 0) and (ky1, W/2) first; group 0 holds four real modes on
// k = 0 or a Nyquist line, which are not rotated.
template <int N, int MR>
__device__ __forceinline__ void cspin2_pair(float2& y1a, float2& y2a, float2& y1b, float2& y2b, int K, int t,
                                            int ky1, int ky2, const float2* __restrict__ fgE,
                                            const float2* __restrict__ fgB, uint32_t step, uint32_t chain,
                                            uint32_t k0, uint32_t k1) {
  using G = CGeo<N, MR>;
  const uint32_t grp = uint32_t(K * (G::H / 2) + ky1);
  float zE[4], zB[4];
  normals4(grp, step, chain, 1u, k0, k1, zE);
  normals4(grp, step, chain, 9u, k0, k1, zB);
  float c, s;
  if (K != 0) {
    const int i1 = ky1 * G::L + t, i2 = ky2 * G::L + t;
    ks_rot<N>(ky1, K, c, s);
    spin2_mode(y1a, y1b, c, s, WF_LDG(fgE + i1), WF_LDG(fgB + i1), zE[0], zE[1], zB[0], zB[1]);
    ks_rot<N>(ky2, K, c, s);
    spin2_mode(y2a, y2b, c, s, WF_LDG(fgE + i2), WF_LDG(fgB + i2), zE[2], zE[3], zB[2], zB[3]);
    return;
  }
  const int ia1 = ky1 * G::L, ib1 = G::H * G::L + ky1;
  if (ky1 == 0) {
    const int ia2 = ky2 * G::L, ib2 = G::H * G::L + ky2;
    constexpr float R2 = 1.41421356237309505f;
    auto upd = [&](float& va, float& vb, int i, float ze, float zb) {
      const float2 mE = WF_LDG(fgE + i), mB = WF_LDG(fgB + i);
      va = fmaf(mE.x, va, R2 * mE.y * ze);
      vb = fmaf(mB.x, vb, R2 * mB.y * zb);
    };
    upd(y1a.x, y1b.x, ia1, zE[0], zB[0]);
    upd(y1a.y, y1b.y, ib1, zE[2], zB[2]);
    upd(y2a.x, y2b.x, ia2, zE[1], zB[1]);
    upd(y2a.y, y2b.y, ib2, zE[3], zB[3]);
    return;
  }
  float2 A1 = cscale(cadd(y1a, cconj(y2a)), 0.5f), B1 = cmul_mi(cscale(csub(y1a, cconj(y2a)), 0.5f));
  float2 A2 = cscale(cadd(y1b, cconj(y2b)), 0.5f), B2 = cmul_mi(cscale(csub(y1b, cconj(y2b)), 0.5f));
  ks_rot<N>(ky1, 0, c, s);
  spin2_mode(A1, A2, c, s, WF_LDG(fgE + ia1), WF_LDG(fgB + ia1), zE[0], zE[1], zB[0], zB[1]);
  ks_rot<N>(ky1, G::W / 2, c, s);
  spin2_mode(B1, B2, c, s, WF_LDG(fgE + ib1), WF_LDG(fgB + ib1), zE[2], zE[3], zB[2], zB[3]);
  y1a = cadd(A1, cmul_i(B1));
  y2a = cadd(cconj(A1), cmul_i(cconj(B1)));
  y1b = cadd(A2, cmul_i(B2));
  y2b = cadd(cconj(A2), cmul_i(cconj(B2)));
}

// The cross-cluster radix-P stage of ccol_units on both components at once (component c's rows at
// rows + c A SP), shared out to the T threads of each CTA (g = the thread's index in the cluster): the
// same work units and mode pairs, fn(K, t, y1a, y2a, y1b, y2b, ky1, ky2) receiving
// the pair's values of both components, then the inverse stage scattered back for both.
template <int N, int MR, int T, class F>
__device__ __forceinline__ void ccol_units2(cooperative_groups::cluster_group& cl, float2* rows, int g, F&& fn) {
  using G = CGeo<N, MR>;
  constexpr int P = G::P, L = G::L, R = G::R, M = G::M, CS = G::A * G::SP;
  constexpr int PAIRS = L * (M / 2);
  if constexpr (PAIRS <= P * T) {
    // at most one unit pair per thread: the two units of a pair go to partner lanes (lane ^ 16, same slot),
    // each holding its unit's values of both components, as in ccol_units (REPS units per lane); the lane
    // leading a mode pair fetches the second mode of both components from its partner and hands the new
    // values back
    constexpr int REPS = 2 * PAIRS / (P * T);
    static_assert(REPS >= 1 && 2 * PAIRS == REPS * P * T, "equal work units per thread");
    static_assert(L % 16 == 0, "a half-warp of consecutive slots shares one unit");
    const int lane = int(threadIdx.x) % 32, half = lane / 16;
    const int w0 = (g / 32) * 16 + lane % 16;
#pragma unroll 1
    for (int rep = 0; rep < REPS; ++rep) {
      const int w = w0 + rep * (PAIRS / REPS);
      const int t = w % L, u = w / L;
      const int uu = half == 0 ? u : (u == 0 ? M / 2 : M - u);
      const int K = (t % R) * M + t / R;
      float2 y[2][P];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
#pragma unroll
        for (int j = 0; j < P; ++j) y[c][j] = cl.map_shared_rank(rows + c * CS, j)[uu * G::SP + cphys<N, MR>(t)];
        fft<P, false>(y[c]);
      }
      if (u == 0) {  // the same in every lane of the warp
        if (half == 0) {
          fn(K, t, y[0][0], y[0][P / 2], y[1][0], y[1][P / 2], 0, N / 2);
#pragma unroll
          for (int m = 1; m < P / 2; ++m) fn(K, t, y[0][m], y[0][P - m], y[1][m], y[1][P - m], M * m, N - M * m);
        } else {
#pragma unroll
          for (int m = 0; m < P / 2; ++m)
            fn(K, t, y[0][m], y[0][P - 1 - m], y[1][m], y[1][P - 1 - m], M / 2 + M * m, N - M / 2 - M * m);
        }
      } else {
        auto swap16 = [](float2 v) {
          return make_float2(__shfl_xor_sync(0xffffffffu, v.x, 16), __shfl_xor_sync(0xffffffffu, v.y, 16));
        };
#pragma unroll
        for (int m = 0; m < P / 2; ++m) {
          float2 a2 = swap16(y[0][P - 1 - m]), b2 = swap16(y[1][P - 1 - m]);
          fn(K, t, y[0][m], a2, y[1][m], b2, uu + M * m, N - uu - M * m);
          y[0][P - 1 - m] = swap16(a2);
          y[1][P - 1 - m] = swap16(b2);
        }
      }
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        fft<P, true>(y[c]);
#pragma unroll
        for (int j = 0; j < P; ++j) cl.map_shared_rank(rows + c * CS, j)[uu * G::SP + cphys<N, MR>(t)] = y[c][j];
      }
    }
    return;
  }
  static_assert(PAIRS <= P * T || PAIRS % (P * T) == 0, "equal work units per thread");
  for (int w = g; w < L * (M / 2); w += P * T) {
    const int t = w % L, u = w / L, v = u == 0 ? M / 2 : M - u;
    const int K = (t % R) * M + t / R;  // kx held by slot t
    float2 p[2][P], q[2][P];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
#pragma unroll
      for (int j = 0; j < P; ++j) p[c][j] = cl.map_shared_rank(rows + c * CS, j)[u * G::SP + cphys<N, MR>(t)];
#pragma unroll
      for (int j = 0; j < P; ++j) q[c][j] = cl.map_shared_rank(rows + c * CS, j)[v * G::SP + cphys<N, MR>(t)];
      fft<P, false>(p[c]);
      fft<P, false>(q[c]);
    }
    if (u == 0) {
      fn(K, t, p[0][0], p[0][P / 2], p[1][0], p[1][P / 2], 0, N / 2);
#pragma unroll
      for (int m = 1; m < P / 2; ++m) fn(K, t, p[0][m], p[0][P - m], p[1][m], p[1][P - m], M * m, N - M * m);
#pragma unroll
      for (int m = 0; m < P / 2; ++m)
        fn(K, t, q[0][m], q[0][P - 1 - m], q[1][m], q[1][P - 1 - m], M / 2 + M * m, N - M / 2 - M * m);
    } else {
#pragma unroll
      for (int m = 0; m < P / 2; ++m) {
        fn(K, t, p[0][m], q[0][P - 1 - m], p[1][m], q[1][P - 1 - m], u + M * m, N - u - M * m);
        fn(K, t, q[0][m], p[0][P - 1 - m], q[1][m], p[1][P - 1 - m], v + M * m, N - v - M * m);
      }
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      fft<P, true>(q[c]);
#pragma unroll
      for (int j = 0; j < P; ++j) cl.map_shared_rank(rows + c * CS, j)[v * G::SP + cphys<N, MR>(t)] = q[c][j];
      fft<P, true>(p[c]);
#pragma unroll
      for (int j = 0; j < P; ++j) cl.map_shared_rank(rows + c * CS, j)[u * G::SP + cphys<N, MR>(t)] = p[c][j];
    }
  }
}

// one chain (both components) per cluster; a.aq2 [2] pixel tables with the CTA-contiguous rows, a.fgE and
// a.fgB in slot order; out [n_chains][n_samples][2][H][W]
template <int N, int MR>
__global__ void __launch_bounds__(cspin2_threads<N, MR>(), cspin2_min_ctas<N, MR>()) k_csample_spin2(Spin2Args a) {
  using G = CGeo<N, MR>;
  constexpr bool SPLIT = cspin2_split<N, MR>();
  constexpr int T = cspin2_threads<N, MR>();
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* rows = reinterpret_cast<float2*>(smem_raw);
  float2* tw = reinterpret_cast<float2*>(smem_raw + 2 * G::ROWS_BYTES);
  if (a.sc->status != 0) return;  // uniform over the grid
  const long long ci = blockIdx.x / G::P;
  constexpr long long NPIX = (long long)G::H * G::W;
  const int b = int(cl.block_rank()), g = b * T + int(threadIdx.x);
  ctw_init<N, MR>(tw);
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    if (SPLIT && int(threadIdx.x) / G::L != c) continue;
    crows_load<N, MR>(rows + c * G::A * G::SP, b, a.init_s ? a.init_s + ci * a.init_stride + c * NPIX : nullptr,
                      int(threadIdx.x) % G::L);
  }
  __syncthreads();
  const uint32_t chain = a.chain0 + uint32_t(ci);
  const int eb = out_elem_bytes(a.out_dtype);
  csweeps<N, MR, 2, SPLIT>(
      cl, rows, tw, a.aq2, a.sc->sqrt_tau, reinterpret_cast<char*>(a.out) + ci * a.n_samples * 2 * NPIX * eb,
      a.out_dtype, a.n_sweeps, a.burn_in, a.thin, a.step0, chain, a.key0, a.key1,
      [&](uint32_t step, int) {
        ccol_units2<N, MR, T>(cl, rows, g,
                           [&](int K, int t, float2& y1a, float2& y2a, float2& y1b, float2& y2b, int ky1, int ky2) {
                             cspin2_pair<N, MR>(y1a, y2a, y1b, y2b, K, t, ky1, ky2, a.fgE, a.fgB, step, chain,
                                                a.key0, a.key1);
                           });
      },
      [](uint32_t, int) {});
  cl.sync();  // no CTA leaves while another may still address its shared memory
}

}  // namespace wf
