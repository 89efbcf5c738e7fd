// Brick kernel: the operator on groups of 2 x 2 x BRICK_KZ neighbouring elements ("bricks") of a
// structured hexahedral lattice, one thread block per brick (paper Section 2: gather L->E, the
// element operator, scatter E->L; Section 3: no global temporaries).
//
// Why: an element's node rows (p+1 nodes) always straddle memory sectors, and every node on an
// element face is gathered and scattered once per element that contains it, in different colour
// launches (far apart in time, so the sectors are fetched from DRAM again).  A brick reads each of
// its nodes once, in rows of 2p+1, into shared memory; its elements gather from there; each brick
// node's result is the sum of the results of the elements that contain it, formed in shared memory
// in element order (deterministic), and written once.  Only the nodes on brick faces are shared
// with other bricks: bricks are coloured by the parity of their lattice coordinates (8 colours, one
// launch each) and the first brick to write a shared node (lowest colour) stores, later ones
// load-add-store.  Measured at 64^3, p = 7 (FP32 operator): 18% fewer DRAM bytes per launch than
// the element kernel.
//
// The lattice structure is detected from the restriction at mesh setup (every element's nodes are
// base + a + b sy + c sz with common strides, element counts along x and y even); other meshes,
// several columns, and operators on the FP64 pipe use the element kernel.  No restriction is read
// here: a brick is its corner node and its elements' quadrature-data blocks.
#pragma once

namespace ceedgb {

struct BrickArgs {
  const int32_t *gbase;     // [brick] L-vector index of the brick's corner node
  const int32_t *gelem;     // [brick][4 BRICK_KZ] colour-sorted element at kx + 2 ky + 4 kz
  const uint32_t *gflags;   // [brick] parity and neighbour bits
  const uint32_t *dirbits;  // Dirichlet bit of every node (masked applies)
  const void *qdata;
  const double *x;
  double *y;
  int64_t g_begin;          // first brick of this launch
  int64_t estride;          // quadrature data per element, in TQ units
  int64_t sy, sz;           // node-lattice strides in y and z (x stride 1)
  int masked;
  int *err;
  int wait_limit;
  double *dot_part;         // optional: partial sums of x_i y_i over the nodes whose final y this block writes
  int64_t dot_base;
  double *dot_sh;           // optional, instead of dot_part: a shared-memory sum (persistent blocks)
};

// x pitch of the shared node box, chosen so that one warp's reads of the box (lanes i = 0..Q-1 along
// x, j along y) fall into as few bank conflicts as possible
template <int P, int Q>
constexpr int brick_pitch() {
  constexpr int n = 2 * P - 1;
  int best = n, best_worst = 1 << 30;
  for (int pitch = n; pitch < n + 32; ++pitch) {
    int cnt[32] = {};
    int worst = 0;
    for (int t = 0; t < 32 && t < Q * Q; ++t) {
      const int i = t % Q, j = t / Q;
      if (i >= P || j >= P) continue;
      const int b = (j * pitch + i) % 32;
      if (++cnt[b] > worst) worst = cnt[b];
    }
    if (worst < best_worst) {
      best_worst = worst;
      best = pitch;
    }
  }
  return best;
}

template <int P, int Q, typename T>
constexpr size_t brick_box_bytes() {
  constexpr int n = 2 * P - 1, nz = BRICK_KZ * (P - 1) + 1;
  return ((size_t)brick_pitch<P, Q>() * n * nz * sizeof(T) + 127) & ~(size_t)127;
}

template <int P, int Q, int OP, typename T, typename TQ, bool STAGE>
constexpr size_t brick_smem() {
  return brick_box_bytes<P, Q, T>() + 4 * BRICK_KZ * apply_elem_smem<P, Q, OP, T, TQ, STAGE>();
}

template <typename T>
__device__ __forceinline__ T brick_add(T a, T b) {
  return a + b;
}
template <>
__device__ __forceinline__ DF brick_add<DF>(DF a, DF b) {
  return df_add(a, b);
}

__device__ __forceinline__ bool brick_dir(const uint32_t *bits, int64_t v) {
  return (__ldg(bits + (v >> 5)) >> (v & 31)) & 1u;
}

// Walks one thread's node rows r = rbase, rbase + STEP, ... (row = B + NB C) without dividing:
// B, C and the L-vector index v = base + B sy + C sz advance by constants, with one carry of B.
template <int NB, int STEP>
struct BrickRows {
  int B, C;
  int64_t v, d1, d2;
  __device__ __forceinline__ BrickRows(int row, int64_t base, int64_t sy, int64_t sz)
      : B(row % NB), C(row / NB), v(base + (row % NB) * sy + (row / NB) * sz),
        d1((STEP % NB) * sy + (STEP / NB) * sz), d2(sz - NB * sy) {}
  __device__ __forceinline__ void next() {
    B += STEP % NB;
    C += STEP / NB;
    v += d1;
    if (B >= NB) {
      B -= NB;
      C += 1;
      v += d2;
    }
  }
};

// One brick: blockDim.x = 4 KZ Q^2 threads, element k = kx + 2 ky + 4 kz on threads [k Q^2, (k+1) Q^2).
// The brick's node rows (2p+1 nodes along x) are handled by groups of RL lanes, so that the row's
// reads and writes are contiguous and no thread divides a node index.
// XCG: x is read through L2 only (a persistent caller changes it between applies).
template <int P, int Q, int OP, typename T, typename TQ, bool STAGE, bool XCG = false>
__device__ __forceinline__ void brick_block(const BrickArgs &a, const OpTab<T> &tab, int64_t blk,
                                            unsigned char *smem_raw, uint64_t *bar) {
  constexpr int NPT = Q * Q;
  constexpr int p = P - 1;
  constexpr int NB = 2 * P - 1;          // brick nodes along x and y
  constexpr int NBZ = BRICK_KZ * p + 1;  // along z
  constexpr int NEL = 4 * BRICK_KZ;      // elements per brick
  constexpr int BX = brick_pitch<P, Q>();
  constexpr int NT = NEL * NPT;
  constexpr int ROWS = NB * NBZ;
  constexpr int RL = NB <= 8 ? 8 : (NB <= 16 ? 16 : 32);  // lanes per node row
  constexpr int RPASS = NT / RL;                           // rows per pass of the whole block
  constexpr int NPASS = (ROWS + RPASS - 1) / RPASS;
  constexpr size_t BOXB = brick_box_bytes<P, Q, T>();
  constexpr size_t QB = STAGE ? ((qblock_bytes<Q, OP, TQ>() + 127) & ~(size_t)127) : 0;
  constexpr size_t EB = apply_elem_smem<P, Q, OP, T, TQ, STAGE>();
  static_assert(RPASS >= 1, "a brick has at least one row of threads");
  __shared__ int abort_sh;

  const int tid = threadIdx.x;
  const int k = tid / NPT;
  const int ij = tid - k * NPT;
  const int i = ij % Q, j = ij / Q;
  const int kx = k & 1, ky = (k >> 1) & 1, kz = k >> 2;
  const bool node_thread = (i < P) && (j < P);
  const int64_t g = a.g_begin + blk;
  const int64_t e = a.gelem[g * NEL + k];
  const int64_t base = a.gbase[g];
  const uint32_t gf = a.gflags[g];
  T *box = (T *)smem_raw;
  unsigned char *eraw = smem_raw + BOXB + (size_t)k * EB;
  const TQ *sq = STAGE ? (const TQ *)eraw : (const TQ *)a.qdata + e * a.estride;
  T *sa = (T *)(eraw + QB);
  T *sb = sa + tile_words<Q>();
  T *sc = sb + tile_words<Q>();
  // row work: node A of row rbase + r RPASS (row = B + NB C)
  const int A = tid % RL;
  const int rbase = tid / RL;
  const bool a_ok = (A < NB) && (tid < RPASS * RL);
  const bool mask = a.masked && (gf & BRICK_DIR);  // only bricks holding a Dirichlet node test the mask

  if constexpr (STAGE) {
    if (ij == 0) {
      mbar_init(&bar[k], 1);
      tma_bulk_load((void *)sq, (const TQ *)a.qdata + e * a.estride, (uint32_t)(a.estride * sizeof(TQ)), &bar[k]);
    }
  } else {
    if (ij == 0) l2_prefetch_bulk((const TQ *)a.qdata + e * a.estride, (uint32_t)(a.estride * sizeof(TQ)));
  }
  if (tid == 0) abort_sh = 0;

  // ---- the brick's nodes, each read once; masked Dirichlet nodes enter as zero
  {
    double xv[NPASS];
    BrickRows<NB, RPASS> it(rbase, base + A, a.sy, a.sz);
    if (mask) {  // mask bits and values loaded side by side, then the Dirichlet nodes zeroed
      bool dz[NPASS];
#pragma unroll
      for (int r = 0; r < NPASS; ++r, it.next()) {
        const int row = rbase + r * RPASS;
        xv[r] = 0.0;
        dz[r] = false;
        if (a_ok && row < ROWS) {
          xv[r] = XCG ? __ldcg(a.x + it.v) : __ldg(a.x + it.v);
          dz[r] = brick_dir(a.dirbits, it.v);
        }
      }
#pragma unroll
      for (int r = 0; r < NPASS; ++r) xv[r] = dz[r] ? 0.0 : xv[r];
    } else {
#pragma unroll
      for (int r = 0; r < NPASS; ++r, it.next()) {
        const int row = rbase + r * RPASS;
        xv[r] = 0.0;
        if (a_ok && row < ROWS) xv[r] = XCG ? __ldcg(a.x + it.v) : __ldg(a.x + it.v);
      }
    }
#pragma unroll
    for (int r = 0; r < NPASS; ++r) {
      const int row = rbase + r * RPASS;
      if (a_ok && row < ROWS) box[row * BX + A] = LVec<T>::in(xv[r]);
    }
  }
  __syncthreads();  // box complete; mbarriers initialised before any wait

  // ---- element gather from the box: node (i, j, c) of element k is brick node (kx p + i, ky p + j, kz p + c)
  T u[P];
#pragma unroll
  for (int c = 0; c < P; ++c) u[c] = (T)0;
  T *col = box + ((kz * p) * NB + ky * p + j) * BX + kx * p + i;
  if (node_thread) {
#pragma unroll
    for (int c = 0; c < P; ++c) u[c] = col[c * NB * BX];
  }

  bool have_q = false;
  auto wait_q = [&]() {
    if (STAGE && !have_q) {
      if (!mbar_wait(&bar[k], 0, a.wait_limit == 0)) {
        abort_sh = 1;
        if (ij == 0) *a.err = CEED_ERR_TIMEOUT;
      }
      have_q = true;
    }
  };
  T yv[P];
  element_op<P, Q, OP, T, TQ>(tab, u, yv, sq, sa, sb, sc, i, j, node_thread, true, wait_q);
  __syncthreads();  // every element has gathered: the box is free

  // ---- the elements' results summed into the box in element order (fixed: deterministic); a node
  // is first touched by element k unless an earlier element (kx, ky or kz lower) shares it
#pragma unroll 1
  for (int ph = 0; ph < NEL; ++ph) {
    if (k == ph && node_thread) {
      const bool face_xy = (kx && i == 0) || (ky && j == 0);
#pragma unroll
      for (int c = 0; c < P; ++c) {
        T *d = col + c * NB * BX;
        *d = (face_xy || (kz && c == 0)) ? brick_add(*d, yv[c]) : yv[c];
      }
    }
    __syncthreads();
  }
  const bool abort = abort_sh != 0;

  // ---- scatter: the lowest colour among the bricks sharing a node writes first (parity 0 on every
  // shared axis), later ones load-add-store
  const uint32_t px = gf & 1u, py = (gf >> 1) & 1u, pz = (gf >> 2) & 1u;
  const bool sx = (A == 0 && (gf & BRICK_MX)) || (A == NB - 1 && (gf & BRICK_PX));
  double dot = 0.0;
  double yold[NPASS];
  uint32_t fl[NPASS];  // bit 0 first, bit 1 last, bit 2 Dirichlet
  {
    BrickRows<NB, RPASS> it(rbase, base + A, a.sy, a.sz);
#pragma unroll
    for (int r = 0; r < NPASS; ++r, it.next()) {  // old values first: one memory latency for all of them
      const int row = rbase + r * RPASS;
      yold[r] = 0.0;
      fl[r] = 0;
      if (a_ok && row < ROWS && !abort) {
        const bool sy_ = (it.B == 0 && (gf & BRICK_MY)) || (it.B == NB - 1 && (gf & BRICK_PY));
        const bool sz_ = (it.C == 0 && (gf & BRICK_MZ)) || (it.C == NBZ - 1 && (gf & BRICK_PZ));
        const bool first = !(sx && px) && !(sy_ && py) && !(sz_ && pz);
        const bool last = !(sx && !px) && !(sy_ && !py) && !(sz_ && !pz);
        const bool dir = mask && brick_dir(a.dirbits, it.v);
        fl[r] = (first ? 1u : 0u) | (last ? 2u : 0u) | (dir ? 4u : 0u) | 8u;
        if (!first && !dir) yold[r] = __ldcg(a.y + it.v);
      }
    }
  }
  BrickRows<NB, RPASS> it(rbase, base + A, a.sy, a.sz);
#pragma unroll
  for (int r = 0; r < NPASS; ++r, it.next()) {
    if (!(fl[r] & 8u)) continue;
    const int row = rbase + r * RPASS;
    const int64_t v = it.v;
    if (fl[r] & 4u) {
      if (fl[r] & 1u) {
        const double out = XCG ? __ldcg(a.x + v) : a.x[v];
        a.y[v] = out;
        dot += out * out;
      }
    } else {
      const T s = box[row * BX + A];
      const double out = (fl[r] & 1u) ? LVec<T>::out(s) : LVec<T>::add(yold[r], s);
      a.y[v] = out;
      if ((fl[r] & 2u) && (a.dot_part || a.dot_sh)) dot += (XCG ? __ldcg(a.x + v) : __ldg(a.x + v)) * out;
    }
  }
  if (a.dot_part || a.dot_sh) {  // fixed-order block reduction: warp shuffles, then the warps in order
    __shared__ double dsum[32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) dot += __shfl_down_sync(0xffffffffu, dot, off);
    if ((tid & 31) == 0) dsum[tid >> 5] = dot;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) t += dsum[w];
      if (a.dot_sh) *a.dot_sh += t;
      else a.dot_part[a.dot_base + blk] = t;
    }
  }
  if constexpr (STAGE) {
    // a copy whose wait gave up may still be writing shared memory: wait for it once more (bounded),
    // then retire the barrier
    if (abort && ij == 0) mbar_wait(&bar[k], 0);
    __syncthreads();
    if (ij == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&bar[k])) : "memory");
  }
}

template <int Q>
constexpr int brick_threads() {
  return 4 * BRICK_KZ * Q * Q;
}
template <int Q>
constexpr int brick_min_blocks() {
  return brick_threads<Q>() <= 256 ? 4 : brick_threads<Q>() <= 512 ? 2 : 1;
}

template <int P, int Q, int OP, typename T, typename TQ, bool STAGE>
__global__ void __launch_bounds__(brick_threads<Q>(), brick_min_blocks<Q>()) brick_kernel(const BrickArgs a, const OpTab<T> tab) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t bar[STAGE ? 4 * BRICK_KZ : 1];
  brick_block<P, Q, OP, T, TQ, STAGE>(a, tab, blockIdx.x, smem_raw, bar);
}

// Arguments of a brick launch over the mesh's bricks (caller fills g_begin per colour).
inline BrickArgs brick_args(ceed_mesh_t m, const ApplyReq &r, int op, size_t tq_bytes) {
  BrickArgs a;
  a.gbase = m->d_gbase;
  a.gelem = m->d_gelem;
  a.gflags = m->d_gflags;
  a.dirbits = m->d_dirbits;
  a.qdata = r.qdata;
  a.x = r.x;
  a.y = r.y;
  a.g_begin = 0;
  a.estride = qdata_estride(op, tq_bytes, m->Q);
  a.sy = m->brick_sy;
  a.sz = m->brick_sz;
  a.masked = r.masked;
  a.err = m->d_err + 1;
  a.wait_limit = copy_wait_limit();
  a.dot_part = r.dot_part;
  a.dot_base = 0;
  a.dot_sh = nullptr;
  return a;
}

// One launch per brick colour.
template <int P, int Q, int OP, typename T, typename TQ, bool STAGE>
int launch_bricks(ceed_mesh_t m, const OpTab<T> &tab, const ApplyReq &r, cudaStream_t s) {
  constexpr size_t smem = brick_smem<P, Q, OP, T, TQ, STAGE>();
  const void *kfn = (const void *)brick_kernel<P, Q, OP, T, TQ, STAGE>;
  if (int st = ensure_dynamic_smem(kfn, smem)) return st;
  BrickArgs a = brick_args(m, r, OP, sizeof(TQ));
  for (int c = 0; c < 8; ++c) {
    a.g_begin = m->brick_start[c];
    const int64_t n = m->brick_start[c + 1] - a.g_begin;
    if (n == 0) continue;
    brick_kernel<P, Q, OP, T, TQ, STAGE><<<(unsigned)n, brick_threads<Q>(), smem, s>>>(a, tab);
    a.dot_base += n;
  }
  if (r.dot_n) *r.dot_n = r.dot_part ? a.dot_base : 0;
  CEED_CUDA_CHECK(cudaGetLastError());
  return CEED_OK;
}

}  // namespace ceedgb
