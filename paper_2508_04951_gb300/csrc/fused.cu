// Cluster-fused FFT correction kernels; see fused.cuh for the data flow.
#include <algorithm>
#include <cooperative_groups.h>

#include "fused.cuh"
#include "tma.cuh"

namespace cg = cooperative_groups;

namespace dc {

namespace {

constexpr int kRowN = 4096;             // row length
constexpr int kRowThreads = 256;        // threads per row (one radix-16 butterfly each)
constexpr int kRowPitch = kRowN + kRowN / 16;

DC_DEV int pad16(int p) { return p + (p >> 4); }

// Stage twiddles of a 4096-point row from the precomputed tables: stage 2
// multiplies v[r] by W256^(r k), k = j mod 16; stage 3 by W4096^(r j).  Only
// the table rows r = 1, 2, 4, 8 are read (coalesced across the warp); the
// other powers are their products (apply_powers).  The one-buffer rows load
// the bases ahead of the CTA barrier that precedes their use; the two-buffer
// row of the single-CTA transform takes them loaded at kernel start.
template <int DIR>
DC_DEV void stage2_bases(float2 (&b)[4], const float2* __restrict__ tw, int k) {
  const float2* t = tw + kTwS2 + k;             // row r at (r - 1) * 16
  b[0] = conj_if<DIR>(__ldg(t));
  b[1] = conj_if<DIR>(__ldg(t + 16));
  b[2] = conj_if<DIR>(__ldg(t + 48));
  b[3] = conj_if<DIR>(__ldg(t + 112));
}
template <int DIR>
DC_DEV void stage3_bases(float2 (&b)[4], const float2* __restrict__ tw, int j) {
  const float2* t = tw + kTwS3 + j;             // row r at (r - 1) * 256
  b[0] = conj_if<DIR>(__ldg(t));
  b[1] = conj_if<DIR>(__ldg(t + 256));
  b[2] = conj_if<DIR>(__ldg(t + 768));
  b[3] = conj_if<DIR>(__ldg(t + 1792));
}

// One 4096-point row, thread j of 256.  In: v[r] = x[j + 256 r].
// Out: v[r] = X[j + 256 r].  Three radix-16 Stockham stages exchanging
// through two padded shared-memory buffers (element p at p + p/16): stage 1
// writes b1, stage 2 reads b1 and writes b2, stage 3 reads b2.  One CTA
// barrier per exchange; the caller must make sure nobody still reads b1 when
// this starts.  Every thread of the CTA calls this together.  f2, f3: the
// forward transform's stage bases (stage2_bases / stage3_bases with DIR =
// -1), loaded by the caller ahead of time; the inverse takes their
// conjugates.
template <int DIR>
DC_DEV void row4096(float2 (&v)[16], float2* b1, float2* b2, int j, const float2 (&f2)[4],
                    const float2 (&f3)[4]) {
  float2 w[4];
  dft16<DIR>(v);                                           // Ns = 1
#pragma unroll
  for (int r = 0; r < 16; ++r) b1[pad16(16 * j + r)] = v[r];
#pragma unroll
  for (int b = 0; b < 4; ++b) w[b] = conj_if<DIR>(f2[b]);
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = b1[pad16(j + 256 * r)];
  apply_powers<16>(v, w);                                  // Ns = 16: W256^(r k)
  dft16<DIR>(v);
  const int base = (j >> 4) * 256 + (j & 15);
#pragma unroll
  for (int r = 0; r < 16; ++r) b2[pad16(base + 16 * r)] = v[r];
#pragma unroll
  for (int b = 0; b < 4; ++b) w[b] = conj_if<DIR>(f3[b]);
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = b2[pad16(j + 256 * r)];
  apply_powers<16>(v, w);                                  // Ns = 256: W4096^(r j)
  dft16<DIR>(v);
}

// One 4096-point row, thread j of 256.  In: v[r] = x[j + 256 r].
// Out: v[r] = X[j + 256 r].  Three radix-16 Stockham stages with the data in
// registers, exchanging through one padded shared-memory buffer (element p
// at p + p/16): a CTA barrier after each exchange's writes and one before
// the second exchange's writes.  The caller must make sure nobody still
// reads b when this starts; on
// return other threads may still be reading b.  Every thread of the CTA
// calls this together.
template <int DIR>
DC_DEV void row4096_1buf(float2 (&v)[16], float2* b, int j, const float2* __restrict__ tw) {
  float2 w[4];
  dft16<DIR>(v);
#pragma unroll
  for (int r = 0; r < 16; ++r) b[pad16(16 * j + r)] = v[r];
  stage2_bases<DIR>(w, tw, j & 15);
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = b[pad16(j + 256 * r)];
  apply_powers<16>(v, w);
  dft16<DIR>(v);
  const int base = (j >> 4) * 256 + (j & 15);
  stage3_bases<DIR>(w, tw, j);
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 16; ++r) b[pad16(base + 16 * r)] = v[r];
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = b[pad16(j + 256 * r)];
  apply_powers<16>(v, w);
  dft16<DIR>(v);
}

// row4096_1buf with the stage bases read from shared-memory copies of the
// table rows r = 1, 2, 4, 8 (s2: [4][16] of W256^(r k), s3: [4][256] of
// W4096^(r j), forward values as in the table): a persistent kernel copies
// them once, and the row's base loads then neither miss L1 nor wait on L2.
template <int DIR>
DC_DEV void row4096_1buf_sm(float2 (&v)[16], float2* b, int j, const float2* s2, const float2* s3) {
  float2 w[4];
  dft16<DIR>(v);
#pragma unroll
  for (int r = 0; r < 16; ++r) b[pad16(16 * j + r)] = v[r];
#pragma unroll
  for (int q = 0; q < 4; ++q) w[q] = conj_if<DIR>(s2[q * 16 + (j & 15)]);
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = b[pad16(j + 256 * r)];
  apply_powers<16>(v, w);                                  // Ns = 16: W256^(r k)
  dft16<DIR>(v);
  const int base = (j >> 4) * 256 + (j & 15);
#pragma unroll
  for (int q = 0; q < 4; ++q) w[q] = conj_if<DIR>(s3[q * 256 + j]);
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 16; ++r) b[pad16(base + 16 * r)] = v[r];
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = b[pad16(j + 256 * r)];
  apply_powers<16>(v, w);                                  // Ns = 256: W4096^(r j)
  dft16<DIR>(v);
}

// row4096_1buf, and once every thread has read the buffer for the last time
// (before the last stage's twiddles and DFT) the cluster barrier is arrived
// at with release semantics: peers may overwrite the buffer after their wait,
// while this CTA still finishes its last stage.
template <int DIR>
DC_DEV void row4096_1buf_arrive(float2 (&v)[16], float2* b, int j, const float2* __restrict__ tw) {
  float2 w[4];
  dft16<DIR>(v);
#pragma unroll
  for (int r = 0; r < 16; ++r) b[pad16(16 * j + r)] = v[r];
  stage2_bases<DIR>(w, tw, j & 15);
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = b[pad16(j + 256 * r)];
  apply_powers<16>(v, w);
  dft16<DIR>(v);
  const int base = (j >> 4) * 256 + (j & 15);
  stage3_bases<DIR>(w, tw, j);
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 16; ++r) b[pad16(base + 16 * r)] = v[r];
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = b[pad16(j + 256 * r)];
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  apply_powers<16>(v, w);
  dft16<DIR>(v);
}

// One 4096-point row with a single CTA barrier, thread j of 256.  In:
// v[p] = x[256 p + j].  Out: v[b] = X[hw_sigma(j) + 256 b].
// The four-step split 4096 = 16 x 256 (n = 256 p + q, k = s + 16 t):
//   X[s + 16 t] = sum_q W256^(q t) [W4096^(q s) sum_p x[256 p + q] W16^(p s)]
// -- thread q takes the length-16 DFT over p and the twiddle W4096^(q s);
// one CTA-wide exchange gives half-warp s the 256 values of sub-problem s;
// its length-256 DFT (256 = 16 x 16: q = 16 u + w, t = a + 16 b) takes a
// length-16 DFT over u in thread w, the twiddle W256^(w a), a 16 x 16
// transpose inside the half-warp (shared memory, __syncwarp only) and a
// length-16 DFT over w in thread a.  Half-warp s only ever touches its own
// 272-element region of b after the barrier, so the transpose needs no CTA
// barrier.  ARRIVE: arrive at the cluster barrier (release) once this
// thread's last read of b is done.  The caller must make sure nobody still
// reads b when this starts; on return other threads may still read b.
DC_DEV int hw_sigma(int j) { return (j >> 4) + ((j & 15) << 4); }

// Where a received row keeps column c (c < COLS) of the column owner:
// rpos(c) = 256 (c >> 8) + sw16(hw_sigma(c & 255)), sw16(x) = x ^ ((x >> 4)
// & 15).  The half-warp row leaves column hw_sigma(j) + 256 m in thread j,
// which so stores at 256 m + sw16(j): a warp's 32 remote stores fill one
// 256-byte block (the XOR only permutes inside each 16-element group), the
// form the distributed-shared-memory path moves fastest (scattered
// addresses cost far more), while the owner's lanes, reading columns
// 16 h + a (+ 256 p) at 16 a + (h ^ a), meet 16 different bank pairs.
DC_DEV int sw16(int x) { return x ^ ((x >> 4) & 15); }
DC_DEV int rpos(int c) { return (c & ~255) + sw16(hw_sigma(c & 255)); }

template <int DIR, bool ARRIVE>
DC_DEV void row4096_hw(float2 (&v)[16], float2* b, int j, const float2* __restrict__ tw) {
  float2 w[4];
  stage3_bases<DIR>(w, tw, j);                             // issued ahead of the DFT
  dft16<DIR>(v);                                           // over p
  apply_powers<16>(v, w);                                  // W4096^(q s), q = j
#pragma unroll
  for (int r = 0; r < 16; ++r) b[pad16(256 * r + j)] = v[r];
  const int s = j >> 4, t = j & 15;
  stage2_bases<DIR>(w, tw, t);
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 16; ++u) v[u] = b[pad16(256 * s + 16 * u + t)];   // q = 16 u + w, w = t
  dft16<DIR>(v);                                           // over u
  apply_powers<16>(v, w);                                  // W256^(w a)
  float2* reg = b + 272 * s;                               // = pad16(256 s): the half-warp's region
  __syncwarp();                                            // its reads of the region are done
#pragma unroll
  for (int a = 0; a < 16; ++a) reg[17 * a + t] = v[a];     // V[w][a]
  __syncwarp();
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = reg[17 * t + q];     // thread a = t: V[w = q][a]
  if constexpr (ARRIVE) asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  dft16<DIR>(v);                                           // over w
}

// The per-bin factors of the full correction on 16 bins k0 + s i held by one
// thread: the caller's table (I.ptab, in the four-step layout, entries
// t0 .. t0 + 15: exp(-i phi_k) times anything else the call bundles into the
// frequency domain, e.g. a matched filter's conjugate replica spectrum) when
// there is one, else exp(-i phi_k) of Eq. 16 from the phase constants.
DC_DEV void bin_factors(const FftItem& I, int k0, int s, int t0, float2 (&u)[16]) {
  if (I.ptab) {
    const float4* t = reinterpret_cast<const float4*>(I.ptab + t0);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float4 w = __ldg(t + i);
      u[2 * i] = cmul(u[2 * i], make_float2(w.x, w.y));
      u[2 * i + 1] = cmul(u[2 * i + 1], make_float2(w.z, w.w));
    }
  } else {
    iono_apply_run16(I.ph, k0, s, u);
  }
}

// Wait half of a split cluster barrier (acquire), after an arrive.release.
template <int CL> DC_DEV void cluster_wait() {
  if constexpr (CL > 1) asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Transform p of a FUSED_APPLY launch: from the item list, or formed from
// the grid description (FusedArgs::grid_src).
DC_DEV FftItem apply_item(const FusedArgs& a, int p) {
  if (!a.grid_src) return a.items[p];
  FftItem I = {};
  const int i = p / a.grid_n_tec, t = p - i * a.grid_n_tec;
  const size_t L = (size_t)1 << a.log2L;
  I.src = a.grid_src + (size_t)i * L;
  I.ptab = a.grid_ptab + (size_t)t * L;
  I.dst = a.grid_dst + (size_t)p * a.grid_n_out;
  I.n_valid = a.grid_n_out;
  I.n_out = a.grid_n_out;
  return I;
}

// Spectra (FUSED_SPEC): one row k1 of the four-step spectrum per CTA, one
// cluster of L1 CTAs per transform.  Each CTA runs the length-L1 forward
// DFTs of its 4096 / L1 columns straight from global memory, applies
// W_L^(n2 k1) and writes element k1 of column n2 into the shared memory of
// the CTA owning row k1 (plain remote stores between two cluster barriers:
// every peer running before, every column delivered after); the received
// row is transformed in the same buffer.
template <int LOG2L1>
__global__ void __launch_bounds__(kRowThreads, 4) spec_kernel(FusedArgs a) {
  constexpr int L1 = 1 << LOG2L1;
  constexpr int COLS = kRowN / L1;              // columns per CTA
  constexpr int PER = COLS / kRowThreads;       // columns per thread
  extern __shared__ __align__(128) float2 sm[];
  float2* A = sm;                               // [kRowPitch] received row, row FFT buffer
  const int k1 = L1 > 1 ? (int)cg::this_cluster().block_rank() : 0;
  const FftItem I = a.items[blockIdx.x >> LOG2L1];
  const int j = threadIdx.x;
  float2 v[16];
  if constexpr (L1 == 1) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int n = j + 256 * r;
      v[r] = n < I.n_valid ? __ldg(I.src + n) : make_float2(0.f, 0.f);
    }
  } else {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");   // this CTA runs
    const float2* T = a.t4 + kT4Offset(L1);
#pragma unroll
    for (int p = 0; p < PER; ++p) {
      const int n2 = k1 * COLS + j + 256 * p;
      float2 col[L1];
#pragma unroll
      for (int n1 = 0; n1 < L1; ++n1) {
        const int n = n2 + kRowN * n1;
        col[n1] = n < I.n_valid ? __ldg(I.src + n) : make_float2(0.f, 0.f);
      }
      dft<L1, -1>(col);
      float2 w[4];                              // W_L^(2^b n2), conjugates of the table rows
#pragma unroll
      for (int b = 0; b < LOG2L1; ++b) w[b] = conj_if<+1>(__ldg(T + b * kRowN + n2));
      apply_powers<L1>(col, w);
      if (p == 0) cluster_wait<L1>();           // every peer runs: its shared memory exists
      const uint32_t dst = smem_addr(A + pad16(n2));
#pragma unroll
      for (int q = 0; q < L1; ++q) st_cluster_c64(dsmem_map(dst, q), col[q]);
    }
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");   // columns delivered
    cluster_wait<L1>();
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = A[pad16(j + 256 * r)];
    __syncthreads();                            // the row FFT overwrites A
  }
  row4096_1buf<-1>(v, A, j, a.tw);
#pragma unroll
  for (int r = 0; r < 16; ++r) I.dst[(size_t)k1 * kRowN + j + 256 * r] = v[r];
}

template <int LOG2L1>
cudaError_t launch_spec(const FusedArgs& a, cudaStream_t s) {
  constexpr int L1 = 1 << LOG2L1;
  if (L1 > 1 && !a.t4) return cudaErrorInvalidValue;
  const size_t smem = sizeof(float2) * kRowPitch;
  auto k = spec_kernel<LOG2L1>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (L1 > 8) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.n_items * L1));
  cfg.blockDim = dim3(kRowThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = L1;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, a);
}

// Spectrum apply (FUSED_APPLY): G = 2^LOG2G rows of the transform per CTA
// (256 threads per row), one cluster of CL = L1 / G CTAs per transform.  The
// spectrum rows arrive by 32 KiB bulk copies, the phase rows by coalesced
// loads; after the inverse row FFTs each thread writes its 16 outputs X[n2]
// straight into the shared memory of the CTA that owns column n2 (plain
// remote stores), so no CTA reads another's shared memory.  The rows are
// received into the buffers the row FFTs used (one 34 KiB buffer per row,
// 64 registers: 4 / G CTAs per SM): a first cluster barrier after the row
// FFTs frees every buffer, a second one after the stores delivers them.
// The owner then applies W_L^(-n2 q) from the table and runs its columns.
// Two rows per CTA halve the cluster (8 CTAs at L = 65536): fewer peers per
// barrier and exchange, which moves the same bytes faster.
template <int LOG2L1, int LOG2G>
__global__ void __launch_bounds__(kRowThreads << LOG2G, 4 >> LOG2G) apply_kernel(FusedArgs a) {
  constexpr int L1 = 1 << LOG2L1;
  constexpr int G = 1 << LOG2G;                 // rows per CTA
  constexpr int CL = L1 / G;                    // CTAs per transform
  constexpr int NT = kRowThreads * G;
  constexpr int COLS = kRowN / CL;              // columns owned by a CTA
  constexpr int PCOLS = COLS;                   // received rows at rpos(c)
  constexpr int PER = COLS / kRowThreads;       // a row thread's output r goes to CTA r / PER
  constexpr int PERC = COLS / NT;               // columns per thread
  static_assert(G == 1 || CL > 1, "two rows per CTA need a cluster");
  static_assert(G == 1 || L1 * COLS <= G * kRowPitch, "received rows fit the row buffers");
  extern __shared__ __align__(128) float2 sm[];
  float2* R = sm;                               // [L1][PCOLS] received rows (CL > 1), column c
                                                // of row q at q * PCOLS + rpos(c)
  __shared__ __align__(8) unsigned long long bar_in;

  const int rank = CL > 1 ? (int)cg::this_cluster().block_rank() : 0;
  const FftItem I = apply_item(a, blockIdx.x >> (LOG2L1 - LOG2G));
  const int j = threadIdx.x;
  const int h = j / kRowThreads, jj = j % kRowThreads;   // row of the CTA, thread in the row
  const int k1 = rank * G + h;
  float2* A = sm + h * kRowPitch;               // this row's buffer
  if (j == 0) mbar_init(&bar_in, 1);
  __syncthreads();
  if (j == 0) {
    mbar_expect_tx(&bar_in, G * kRowN * sizeof(float2));
#pragma unroll
    for (int g = 0; g < G; ++g)
      bulk_g2s(sm + g * kRowPitch, I.src + (size_t)(rank * G + g) * kRowN, kRowN * sizeof(float2), &bar_in);
  }
  float2 v[16];
  const float2* prow = I.ptab + (size_t)k1 * kRowN;
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = __ldg(prow + jj + 256 * r);
  mbar_wait_bounded(&bar_in, 0, a.err);         // on a timeout: flag raised, keep going
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = cmul(A[jj + 256 * r], v[r]);
  __syncthreads();                              // the row FFT overwrites A
  if constexpr (L1 == 1) row4096_1buf<+1>(v, A, jj, a.tw);
  else row4096_hw<+1, true>(v, A, jj, a.tw);    // arrives at the cluster barrier; v[r] at
                                                // n2 = hw_sigma(jj) + 256 r

  if constexpr (L1 == 1) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int n = j + 256 * r;
      if (n < I.n_out) __stcs(I.dst + n, v[r]);
    }
  } else {
    // every peer's row FFTs are done with their buffers (the release arrive
    // is inside the row FFT)
    cluster_wait<L1>();
    const uint32_t r_loc = smem_addr(R + k1 * PCOLS + sw16(jj));   // rpos(hw_sigma(jj))
    // the farthest element this thread writes in its owners' buffers
    if (DC_IN_BOUNDS(k1 * PCOLS + sw16(jj) + 256 * (PER - 1) < L1 * PCOLS && 16 / PER <= CL, a.err)) {
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int owner = r / PER;              // n2 = hw_sigma(jj) + 256 r -> owner n2 / COLS
        const uint32_t off = (uint32_t)(256 * (r % PER) * sizeof(float2));   // rpos(c + 256 m)
        st_cluster_c64(dsmem_map(r_loc + off, owner), v[r]);
      }
    }
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");   // rows delivered
    const float2* T = a.t4 + kT4Offset(L1);
#pragma unroll
    for (int p = 0; p < PERC; ++p) {
      const int c = j + NT * p;
      const int n2 = rank * COLS + c;
      float2 w[4];
#pragma unroll
      for (int b = 0; b < LOG2L1; ++b) w[b] = __ldg(T + b * kRowN + n2);   // W_L^(-2^b n2)
      if (p == 0) cluster_wait<L1>();           // every peer's stores into R are visible
      float2 col[L1];
#pragma unroll
      for (int q = 0; q < L1; ++q) col[q] = R[q * PCOLS + rpos(c)];
      apply_powers<L1>(col, w);
      dft<L1, +1>(col);
#pragma unroll
      for (int n1 = 0; n1 < L1; ++n1) {
        const int n = n2 + kRowN * n1;
        if (n < I.n_out) __stcs(I.dst + n, col[n1]);
      }
    }
  }
}

template <int LOG2L1, int LOG2G>
cudaError_t launch_apply(const FusedArgs& a, cudaStream_t s) {
  constexpr int L1 = 1 << LOG2L1;
  constexpr int G = 1 << LOG2G;
  constexpr int CL = L1 / G;
  if (L1 > 1 && !a.t4) return cudaErrorInvalidValue;
  const size_t smem = sizeof(float2) * kRowPitch * G;
  auto k = apply_kernel<LOG2L1, LOG2G>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (CL > 8) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.n_items * CL));
  cfg.blockDim = dim3(kRowThreads * G);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, a);
}

// Spectrum apply in two passes through L2 (FUSED_APPLY with a.scratch set):
// no cluster.  A persistent grid takes tasks from one global queue in a
// fixed order.  A row task transforms one 4096-point row of one transform
// (spectrum row times factor row, inverse row) into a scratch slot; a column
// task reads 4096 / L1 columns of one transform back from its slot, applies
// W_L^(-n2 q) and runs the length-L1 inverse columns into the output.  The
// transforms go in chunks of P = a.chunk: the queue alternates the rows of
// chunk i and the columns of chunk i - kApplyLag, and the scratch holds
// (kApplyLag + 2) P transforms (slot = transform mod that), small enough to
// stay in L2 between the passes, so DRAM sees the output once, as with the
// cluster kernel, but no cluster barrier or distributed-shared-memory
// exchange is needed.  A task is counted done by one release reduction
// after a CTA barrier; a column task waits until the L1 rows of its
// transform are counted, a row task until the columns of the slot's
// previous transform are (one thread polls with acquire loads, the others
// wait at a CTA barrier).  The lag keeps both waits on
// tasks queued several blocks earlier (a grid holds about 2.4 blocks of
// tasks at once), so they rarely wait at all.  Every wait is on tasks taken
// from the queue earlier, by CTAs already running, so the order cannot
// deadlock; each wait is bounded (error flag 1 when it runs out, and the
// task goes on).  Counters (a.ctr: queue head, then rows done and columns
// done per transform) start at zero.
constexpr int kApplyLag = kApplyL2Slots - 2;

DC_DEV int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Release add: the writes this thread has made or observed (a CTA barrier
// before it covers the whole CTA's) become visible before the count.
DC_DEV void red_release_gpu(int* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Thread 0: poll *p until it reaches `want`, for about a second at most.
DC_DEV void wait_count(const int* p, int want, int* err) {
  for (int i = 0; i < (1 << 24); ++i) {
    if (ld_acquire_gpu(p) >= want) return;
    __nanosleep(64);
  }
  atomicMax(err, 1);
}

// One task of the two-pass apply as thread 0 decodes it for the CTA.
struct ApplyTask {
  const float2* src;    // the transform's spectrum (row tasks)
  const float2* ptab;   // its factor table (row tasks)
  float2* dst;          // its output (column tasks)
  float2* slot;         // its scratch slot
  int n_out;
  int p;                // transform
  int rq;               // row k1 (row task) or column block q (column task)
  int prev;             // the slot's previous transform, or -1
  int kind;             // 1 row, 2 column, 0 nothing (past the last chunk), -1 queue done
};

template <int LOG2L1>
__global__ void __launch_bounds__(kRowThreads, 4) apply_l2_kernel(FusedArgs a) {
  constexpr int L1 = 1 << LOG2L1;
  constexpr int COLS = kRowN / L1;              // columns of a column task
  constexpr int PER = COLS / kRowThreads;       // columns per thread
  extern __shared__ __align__(128) float2 sm[]; // [kRowPitch] the row buffer
  __shared__ __align__(8) unsigned long long bar_in;
  __shared__ ApplyTask s_ti[2];                 // the task in hand and the next one
  __shared__ float2 s_tw2[64], s_tw3[1024];     // the row's stage-base table rows r = 1, 2, 4, 8
  const int j = threadIdx.x;
  if (j < 64) s_tw2[j] = __ldg(a.tw + kTwS2 + ((1 << (j >> 4)) - 1) * 16 + (j & 15));
#pragma unroll
  for (int q = 0; q < 4; ++q) s_tw3[q * 256 + j] = __ldg(a.tw + kTwS3 + ((1 << q) - 1) * 256 + j);
  const int P = a.chunk;
  const int n_chunks = (a.n_items + P - 1) / P;
  const int per_block = P * L1;                 // the rows (or columns) of one chunk
  // block 2i: rows of chunk i; block 2i + 1: columns of chunk i - kApplyLag
  const int n_tasks = 2 * (n_chunks + kApplyLag) * per_block;
  const int n_slots = (kApplyLag + 2) * P;
  int* head = a.ctr;
  int* row_done = a.ctr + 1;
  int* col_done = a.ctr + 1 + a.n_items;
  const size_t slot_elems = (size_t)L1 * kRowN;
  // thread 0 decodes each task once (the divisions stay off the other threads)
  auto decode = [&](int t) {
    ApplyTask d = {};
    if (t >= n_tasks) {
      d.kind = -1;
      return d;
    }
    const int b = t / per_block, w = t % per_block;
    const bool is_col = b & 1;
    const int chunk = is_col ? (b >> 1) - kApplyLag : b >> 1;
    d.p = chunk * P + w / L1;
    d.rq = w % L1;                              // row k1, or column block q
    if (chunk < 0 || chunk >= n_chunks || d.p >= a.n_items) return d;   // kind 0: nothing
    d.kind = is_col ? 2 : 1;
    const FftItem I = apply_item(a, d.p);
    d.src = I.src;
    d.ptab = I.ptab;
    d.dst = I.dst;
    d.n_out = I.n_out;
    d.slot = a.scratch + (size_t)(d.p % n_slots) * slot_elems;
    d.prev = d.p >= n_slots ? d.p - n_slots : -1;
    return d;
  };
  int t_next = 0;                               // thread 0: the task taken ahead
  if (j == 0) {
    mbar_init(&bar_in, 1);
    s_ti[0] = decode(atomicAdd(head, 1));
  }
  uint32_t phase = 0;
  for (int it = 0;; ++it) {
    __syncthreads();                            // s_ti; the last task's reads of sm are done
    const ApplyTask T = s_ti[it & 1];
    if (T.kind < 0) break;
    if (j == 0) t_next = atomicAdd(head, 1);    // decoded at the end of this task
    const int p = T.p, rq = T.rq;
    if (T.kind > 0 && DC_IN_BOUNDS(rq >= 0 && rq < L1 && p >= 0 && p < a.n_items, a.err)) {
      const bool is_col = T.kind == 2;
      float2* slot = T.slot;
      FftItem I = {};
      I.src = T.src;
      I.ptab = T.ptab;
      I.dst = T.dst;
      I.n_out = T.n_out;
      if (!is_col) {
        if (j == 0) {                           // the spectrum row first: its copy overlaps the rest
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");    // after the last generic reads
          mbar_expect_tx(&bar_in, kRowN * sizeof(float2));
          bulk_g2s(sm, I.src + (size_t)rq * kRowN, kRowN * sizeof(float2), &bar_in);
        }
        float2 v[16];
        const float2* prow = I.ptab + (size_t)rq * kRowN;
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = __ldg(prow + j + 256 * r);
        mbar_wait_bounded(&bar_in, phase, a.err);
        phase ^= 1;
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = cmul(sm[j + 256 * r], v[r]);
        // the slot is free; the CTA barrier orders thread 0's wait before
        // every thread's stores (the others wait there, polling nothing)
        if (j == 0 && T.prev >= 0) wait_count(col_done + T.prev, L1, a.err);
        __syncthreads();                        // also: the row FFT overwrites sm
        row4096_1buf_sm<+1>(v, sm, j, s_tw2, s_tw3);   // v[r] = Y[j + 256 r]
        float2* yrow = slot + (size_t)rq * kRowN;
#pragma unroll
        for (int r = 0; r < 16; ++r) __stcg(yrow + j + 256 * r, v[r]);
        __syncthreads();
        if (j == 0) red_release_gpu(row_done + p, 1);   // every thread's row stores first
      } else {
        const float2* tw4 = a.t4 + kT4Offset(L1);
        float2 w4[PER][4];                      // W_L^(-2^b n2), loaded ahead of the wait
#pragma unroll
        for (int pp = 0; pp < PER; ++pp)
#pragma unroll
          for (int bb = 0; bb < LOG2L1; ++bb) w4[pp][bb] = __ldg(tw4 + bb * kRowN + rq * COLS + j + 256 * pp);
        if (j == 0) wait_count(row_done + p, L1, a.err);
        __syncthreads();
#pragma unroll
        for (int pp = 0; pp < PER; ++pp) {
          const int n2 = rq * COLS + j + 256 * pp;
          float2 col[L1];
#pragma unroll
          for (int q = 0; q < L1; ++q) col[q] = __ldcg(slot + (size_t)q * kRowN + n2);
          apply_powers<L1>(col, w4[pp]);
          dft<L1, +1>(col);
#pragma unroll
          for (int n1 = 0; n1 < L1; ++n1) {
            const int n = n2 + kRowN * n1;
            if (n < I.n_out) __stcs(I.dst + n, col[n1]);
          }
        }
        __syncthreads();
        if (j == 0) red_release_gpu(col_done + p, 1);   // every thread's slot reads first
      }
    }
    if (j == 0) s_ti[(it + 1) & 1] = decode(t_next);
  }
}

template <int LOG2L1>
cudaError_t launch_apply_l2(const FusedArgs& a, cudaStream_t s) {
  if (!a.t4 || !a.scratch || !a.ctr || a.chunk < 1) return cudaErrorInvalidValue;
  const size_t smem = sizeof(float2) * kRowPitch;
  auto k = apply_l2_kernel<LOG2L1>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kRowThreads, smem)) != cudaSuccess)
    return e;
  const long long tasks = 2LL * (a.n_items + (long long)kApplyLag * a.chunk) * (1 << LOG2L1);
  const int grid = (int)std::max(1LL, std::min<long long>((long long)sms * std::max(per_sm, 1), tasks));
  k<<<grid, kRowThreads, smem, s>>>(a);
  return cudaGetLastError();
}

// Full correction (FUSED_FULL): one row k1 of the transform per CTA, one
// cluster of L1 CTAs per transform, one padded buffer per CTA.  The forward
// columns run straight from global memory (zero past n_valid), take
// W_L^(n2 k1) and go to the row owners by plain remote stores; the forward
// row, exp(-i phi_k) / L at bin k1 + L1 k2 (regrouped so that each thread
// owns 16 consecutive k2) and the inverse row follow in the same buffer; the
// inverse row's outputs go to the column owners the same way, which apply
// W_L^(-n2 q) and run the inverse columns (out truncated to n_out).  Cluster
// barriers order it all: every CTA running before the first remote store,
// each exchange delivered before it is read, every buffer free before the
// second exchange overwrites it.  At L = 4096 one CTA holds the whole
// transform and takes two buffers.
template <int LOG2L1>
__global__ void __launch_bounds__(kRowThreads, LOG2L1 == 0 ? 2 : 4) full_kernel(FusedArgs a) {
  constexpr int L1 = 1 << LOG2L1;
  constexpr int COLS = kRowN / L1;              // columns owned by a CTA
  constexpr int PCOLS = COLS;                   // received rows at rpos(c) (as in apply_kernel)
  constexpr int PER = COLS / kRowThreads;       // columns per thread
  constexpr int LOG2L = 12 + LOG2L1;
  extern __shared__ __align__(128) float2 sm[];
  float2* A = sm;                               // [kRowPitch] received row, row FFTs,
  float2* R = sm;                               // then [L1][PCOLS] received inverse rows
  const int k1 = L1 > 1 ? (int)cg::this_cluster().block_rank() : 0;
  const FftItem I = a.items[blockIdx.x >> LOG2L1];
  const int j = threadIdx.x;
  float2 v[16];
  if constexpr (L1 == 1) {
    // L = 4096: one CTA, no exchange; two buffers (a second [kRowPitch]
    // after A) save a CTA barrier per row, which sets this latency path
    float2* B = sm + kRowPitch;
    // every stage base of both rows loaded up front, beside the input: one
    // CTA per transform leaves nothing to hide a load issued per stage
    float2 f2[4], f3[4];
    stage2_bases<-1>(f2, a.tw, j & 15);
    stage3_bases<-1>(f3, a.tw, j);
    pdl_wait();                                 // the input's producer has finished
    // plain loads: a non-coherent load may be scheduled ahead of the wait
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int n = j + 256 * r;
      v[r] = n < I.n_valid ? I.src[n] : make_float2(0.f, 0.f);
    }
    row4096<-1>(v, A, B, j, f2, f3);            // last reads: B after its second barrier
    const bool mult = I.ph.enabled || I.ptab;
    if (mult) {
      // regroup through A (last read before the forward's second barrier)
#pragma unroll
      for (int r = 0; r < 16; ++r) A[pad16(j + 256 * r)] = v[r];
      __syncthreads();
      float2 u[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) u[i] = A[pad16(16 * j + i)];
      bin_factors(I, 16 * j, 1, 16 * j, u);
#pragma unroll
      for (int i = 0; i < 16; ++i) A[pad16(16 * j + i)] = u[i];
      __syncthreads();
#pragma unroll
      for (int r = 0; r < 16; ++r) v[r] = A[pad16(j + 256 * r)];
    }
    const float invL = 1.0f / (float)(1 << LOG2L);
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = cscale(v[r], invL);
    // the inverse row writes first the buffer no thread can still be reading
    if (mult) row4096<+1>(v, B, A, j, f2, f3);
    else row4096<+1>(v, A, B, j, f2, f3);
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int n = j + 256 * r;
      if (n < I.n_out) __stcs(I.dst + n, v[r]);
    }
  } else {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");   // this CTA runs
    const float2* T = a.t4 + kT4Offset(L1);
    pdl_wait();                                 // the input's producer has finished
#pragma unroll
    for (int p = 0; p < PER; ++p) {
      const int n2 = k1 * COLS + j + 256 * p;
      float2 col[L1];
#pragma unroll
      for (int n1 = 0; n1 < L1; ++n1) {
        const int n = n2 + kRowN * n1;
        col[n1] = n < I.n_valid ? I.src[n] : make_float2(0.f, 0.f);   // plain: after pdl_wait
      }
      dft<L1, -1>(col);
      float2 w[4];                              // W_L^(2^b n2), conjugates of the table rows
#pragma unroll
      for (int b = 0; b < LOG2L1; ++b) w[b] = conj_if<+1>(__ldg(T + b * kRowN + n2));
      apply_powers<L1>(col, w);
      if (p == 0) cluster_wait<L1>();           // every peer runs: its shared memory exists
      const uint32_t dst = smem_addr(A + pad16(n2));
#pragma unroll
      for (int q = 0; q < L1; ++q) st_cluster_c64(dsmem_map(dst, q), col[q]);
    }
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");   // columns delivered
    cluster_wait<L1>();
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = A[pad16(j + 256 * r)];
    __syncthreads();                            // the row FFT overwrites A
    row4096_hw<-1, false>(v, A, j, a.tw);      // v[r] = X[hw_sigma(j) + 256 r]
    {
      // back to natural order through A (the inverse row takes v[r] =
      // Y[j + 256 r]), with the factors on runs of 16 bins on the way
      const int sj = hw_sigma(j);
      __syncthreads();                          // every half-warp is done with its region
#pragma unroll
      for (int r = 0; r < 16; ++r) A[pad16(sj + 256 * r)] = v[r];
      __syncthreads();
      if (I.ph.enabled || I.ptab) {
        float2 u[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) u[i] = A[pad16(16 * j + i)];
        bin_factors(I, k1 + L1 * 16 * j, L1, k1 * kRowN + 16 * j, u);
#pragma unroll
        for (int i = 0; i < 16; ++i) A[pad16(16 * j + i)] = u[i];
        __syncthreads();
      }
#pragma unroll
      for (int r = 0; r < 16; ++r) v[r] = A[pad16(j + 256 * r)];
    }
    const float invL = 1.0f / (float)(1 << LOG2L);
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = cscale(v[r], invL);
    __syncthreads();                            // the inverse row writes A first
    row4096_hw<+1, true>(v, A, j, a.tw);        // arrives at the cluster barrier
    cluster_wait<L1>();                         // every peer's buffer is free
    const uint32_t r_loc = smem_addr(R + k1 * PCOLS + sw16(j));    // rpos(hw_sigma(j))
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int owner = r / PER;                // n2 = hw_sigma(j) + 256 r -> owner n2 / COLS
      const uint32_t off = (uint32_t)(256 * (r % PER) * sizeof(float2));   // rpos(c + 256 m)
      st_cluster_c64(dsmem_map(r_loc + off, owner), v[r]);
    }
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");   // rows delivered
#pragma unroll
    for (int p = 0; p < PER; ++p) {
      const int c = j + 256 * p;
      const int n2 = k1 * COLS + c;
      float2 w[4];
#pragma unroll
      for (int b = 0; b < LOG2L1; ++b) w[b] = __ldg(T + b * kRowN + n2);   // W_L^(-2^b n2)
      if (p == 0) cluster_wait<L1>();           // every peer's stores into R are visible
      float2 col[L1];
#pragma unroll
      for (int q = 0; q < L1; ++q) col[q] = R[q * PCOLS + rpos(c)];
      apply_powers<L1>(col, w);
      dft<L1, +1>(col);
#pragma unroll
      for (int n1 = 0; n1 < L1; ++n1) {
        const int n = n2 + kRowN * n1;
        if (n < I.n_out) __stcs(I.dst + n, col[n1]);
      }
    }
  }
}

template <int LOG2L1>
cudaError_t launch_full(const FusedArgs& a, cudaStream_t s) {
  constexpr int L1 = 1 << LOG2L1;
  if (L1 > 1 && !a.t4) return cudaErrorInvalidValue;
  const size_t smem = sizeof(float2) * kRowPitch * (L1 == 1 ? 2 : 1);
  auto k = full_kernel<LOG2L1>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (L1 > 8) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.n_items * L1));
  cfg.blockDim = dim3(kRowThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  // with a.pdl, programmatic serialization: the launch may begin (items,
  // twiddles) while the kernel before it finishes; the kernel waits for it
  // (pdl_wait) before its first read of the input and its first store
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = L1;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  // L = 4096 (one CTA per transform) is no cluster launch
  cfg.attrs = L1 > 1 ? attr : attr + 1;
  cfg.numAttrs = (L1 > 1 ? 1 : 0) + (a.pdl ? 1 : 0);
  return cudaLaunchKernelEx(&cfg, k, a);
}


// Middle pass of the three-pass four-step path for 65536 < L <= 2^20
// (L1 = L / 4096 in 32..256 rows): one 4096-point row per CTA -- forward
// row FFT, exp(-i phi_k) at bin k1 + L1 k2, inverse row FFT, four-step
// twiddle W_L^(-n2 k1) -- in place on the scratch T between the column
// passes.
__global__ void __launch_bounds__(kRowThreads, 4) row_mid_kernel(RowArgs a) {
  extern __shared__ __align__(128) float2 sm[];
  const int L1 = 1 << a.log2L1;
  const int g = blockIdx.x;
  const int item = g >> a.log2L1, k1 = g & (L1 - 1);
  const FftItem I = a.items[item];
  const int j = threadIdx.x;
  float2* bufA = sm;
  const float2* src = I.src + (size_t)k1 * kRowN;
  float2 v[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = src[j + 256 * r];
  row4096_hw<-1, false>(v, bufA, j, a.tw);    // v[r] = X[hw_sigma(j) + 256 r]
  {
    // back to natural order through A, with the factor of bin k = k1 + L1 k2
    // on the way (each thread on 16 consecutive k2)
    const int sj = hw_sigma(j);
    __syncthreads();                           // every half-warp is done with its region
#pragma unroll
    for (int r = 0; r < 16; ++r) bufA[pad16(sj + 256 * r)] = v[r];
    __syncthreads();
    if (I.ph.enabled || I.ptab) {
      float2 u[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) u[i] = bufA[pad16(16 * j + i)];
      bin_factors(I, k1 + L1 * 16 * j, L1, k1 * kRowN + 16 * j, u);
#pragma unroll
      for (int i = 0; i < 16; ++i) bufA[pad16(16 * j + i)] = u[i];
      __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = bufA[pad16(j + 256 * r)];
  }
  __syncthreads();                             // the inverse row writes A first
  row4096_1buf<+1>(v, bufA, j, a.tw);
  if (k1) {
    const float2 a_j = tw_big<+1>(a.tw, (uint32_t)(j * k1), a.log2L);
    const int m16 = 16 * L1 - 1, step = 256 >> a.log2L1;
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = cmul(v[r], cmul(a_j, tw_m<+1>(a.tw, ((r * k1) & m16) * step)));
  }
  float2* dst = I.dst + (size_t)k1 * kRowN;
#pragma unroll
  for (int r = 0; r < 16; ++r) dst[j + 256 * r] = v[r];
}

}  // namespace

cudaError_t launch_row_mid_4096(const RowArgs& a, cudaStream_t s) {
  if (a.n_items <= 0) return cudaSuccess;
  if (a.log2L - a.log2L1 != 12 || a.log2L1 < 5 || a.log2L1 > 8) return cudaErrorInvalidValue;
  const size_t smem = sizeof(float2) * kRowPitch;
  cudaError_t e = cudaFuncSetAttribute(row_mid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  row_mid_kernel<<<(unsigned)(a.n_items << a.log2L1), kRowThreads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fused(int op, const FusedArgs& a, cudaStream_t s) {
  if (a.n_items <= 0) return cudaSuccess;
  switch (op) {
    case FUSED_APPLY:
      switch (a.log2L) {
        case 12: return launch_apply<0, 0>(a, s);
        case 13: return a.scratch ? launch_apply_l2<1>(a, s) : launch_apply<1, 0>(a, s);
        case 14: return a.scratch ? launch_apply_l2<2>(a, s) : launch_apply<2, 0>(a, s);
        case 15: return a.scratch ? launch_apply_l2<3>(a, s)
                       : a.apply_rows2 ? launch_apply<3, 1>(a, s) : launch_apply<3, 0>(a, s);
        case 16: return a.scratch ? launch_apply_l2<4>(a, s)
                       : a.apply_rows2 ? launch_apply<4, 1>(a, s) : launch_apply<4, 0>(a, s);
        default: return cudaErrorInvalidValue;
      }
    case FUSED_FULL:
      switch (a.log2L) {
        case 12: return launch_full<0>(a, s);
        case 13: return launch_full<1>(a, s);
        case 14: return launch_full<2>(a, s);
        case 15: return launch_full<3>(a, s);
        case 16: return launch_full<4>(a, s);
        default: return cudaErrorInvalidValue;
      }
    case FUSED_SPEC:
      switch (a.log2L) {
        case 12: return launch_spec<0>(a, s);
        case 13: return launch_spec<1>(a, s);
        case 14: return launch_spec<2>(a, s);
        case 15: return launch_spec<3>(a, s);
        case 16: return launch_spec<4>(a, s);
        default: return cudaErrorInvalidValue;
      }
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dc
