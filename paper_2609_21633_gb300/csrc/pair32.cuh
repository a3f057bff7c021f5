// FP32 A apply on halo-free tiles with two cells per thread (included by kernels.cu inside its
// namespace, after the tile kernels whose helpers it uses).
//
// Same operator as OpA<float, HG> (Eq. (epsq) then Eq. (localapply) at q_c, Sec. 4, hourglass
// control Eq. (hgstab) when HG), laid out for the FP32 pipe and its packed f32x2 instructions:
//
// * Tiles of 16 x 32 cells, one CTA of 8 warps each; warp w owns the cell rows i0 + 2w and
//   i0 + 2w + 1, lane l the cell column j0 + l.  A thread therefore holds the two cells
//   A = (i, j) and B = (i + 1, j), and every element operation works on both at once: lane x of a
//   float2 is cell A, lane y cell B.  Both cells run the same instruction stream, so the packed
//   arithmetic needs no lane exchange (the wedges are taken one after the other).
// * Node values (the 17 x 36 node patch of a layer per component), the tile's viscosity of a cell
//   layer and the layer constants arrive in shared memory by cp.async, kPAhead layers ahead of the
//   radial sweep in kPStages buffers, so no thread computes global addresses or waits on a global
//   load in the sweep.
// * Cell contributions are summed into node values in a fixed order: the two cells of a thread in
//   registers, the left neighbour's by a warp shuffle, the upper warp's through shared memory.
//   Nodes on the tile lines i = i0, i0 + 16 and j = j0, j0 + 32 leave one float4 partial per tile
//   in the level's ring buffer (the tile-line index of the FP64 halo-free tiles).  k_ring4_fix
//   sums and finishes those inside the diamond, k_ring4_edges those on the diamond edges with the
//   sum over their copies; no atomics, so results do not depend on scheduling.

constexpr int kPTI = 16, kPTJ = 32, kPThreads = 256;  // cells per tile, threads per CTA
constexpr int kPRows = kPTI + 1;                      // node rows i0 .. i0 + 16 of a tile
constexpr int kPRow = 36;                             // staged nodes per row: j0 .. j0 + 35 (33 used)
constexpr int kPNodes = 3 * kPRows * kPRow;           // node values per staged layer
constexpr int kPEta = kPTI * kPTJ * 2;                // viscosity values of the tile's wedges per cell layer
constexpr int kPStage = kPNodes + kPEta;              // floats per stage
constexpr int kPNodeChunks = kPNodes / 4;             // 16-byte copies of the node values of a layer
constexpr int kPStages = 4;                           // staged layers
constexpr int kPAhead = kPStages - 1;                 // layers requested ahead of the bottom one
constexpr int kPExch = 8 * 33;                        // per component: one down-going value per lane + 1
constexpr int kPGeo = 2 * 12;                         // float2 column values per thread: 2 wedges x 12
constexpr int kPMaxKc = 128;                          // cell layers per radial chunk at most
constexpr size_t kPSmemBytes = sizeof(float) * ((size_t)kPStages * kPStage + 2 * 3 * kPExch) +
                               sizeof(float2) * (size_t)kPGeo * kPThreads + sizeof(float4) * (kPMaxKc + 1);
static_assert(kPNodes % 4 == 0 && (kPRows * kPRow) % 4 == 0 && kPRow % 4 == 0 && kPStage % 4 == 0,
              "16-byte staging");
static_assert(kPNodeChunks <= 2 * kPThreads && kPEta / 4 == kPThreads, "copies per thread per layer");
static_assert(kPSmemBytes <= 113 * 1024, "two CTAs per SM");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory");
}

// Per-column data of the two cells, kept in shared memory (the registers hold the radial sweep's
// state): for wedge w at gc[(12 w + q) kPThreads] (the thread's slot), q = 0..8 the M^-1 entries,
// 9 |det M| (times the column factor of 16-bit viscosity), 10 and 11 the eL, eR factors of
// hg_column (hourglass control only).

// One cell layer of the two cells.  tp, bt: the node values at the top and the bottom of the cell
// corners q = 00, 10, 01, 11 (q = 1: i + 1, q = 2: j + 1), per component; with s = top + bottom and
// d = top - bottom, wedge W0 = (00, 10, 01) has a_xi = s_10 - s_00, a_eta = s_01 - s_00,
// a_zeta = d_00 + d_10 + d_01 and W1 = (11, 01, 10) the same with its own node order.  Out: the
// contributions to the bottom and the top node of each corner, except that for corners 00 and 11
// (one wedge each) `bq` holds the bottom contribution negated (it is subtracted by the caller).
// lc: the cell layer's r = w1 / w0, vol w0^2, w0 / (9 w1) and vol w1^2 (layer-table entries 4, 5, 8, 9).
template <bool HG>
__device__ __forceinline__ void pair_cell(const float2 (&tp)[4][3], const float2 (&bt)[4][3], const float2* gc,
                                          const float4 lc, const float2 (&eta)[2], int div_term, float hgk,
                                          float2 (&bq)[4][3], float2 (&tq)[4][3]) {
  const float2 r = p2(lc.x, lc.x), vw2 = p2(lc.y, lc.y);
  float2 A[2][3][3];                        // A[w][c] = (a_xi, a_eta, a_zeta) of wedge w, component c
  float2 D1[HG ? 2 : 1][3], D2[HG ? 2 : 1][3];  // d at a wedge's local nodes 1 and 2 (hourglass control)
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float2 sq[4], dq[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) sq[q] = add2(tp[q][c], bt[q][c]), dq[q] = sub2(tp[q][c], bt[q][c]);
    const float2 d12 = add2(dq[1], dq[2]);
    A[0][c][0] = sub2(sq[1], sq[0]), A[0][c][1] = sub2(sq[2], sq[0]), A[0][c][2] = add2(dq[0], d12);
    A[1][c][0] = sub2(sq[2], sq[3]), A[1][c][1] = sub2(sq[1], sq[3]), A[1][c][2] = add2(dq[3], d12);
    if constexpr (HG) D1[0][c] = dq[1], D2[0][c] = dq[2], D1[HG ? 1 : 0][c] = dq[2], D2[HG ? 1 : 0][c] = dq[1];
  }
  float2 H0[2][3], H1[2][3], Y[2][HG ? 3 : 1][3];  // Y[w][a][c]: top-minus-bottom part at local node a
#pragma unroll
  for (int w = 0; w < 2; ++w) {
    float2 M[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) M[q] = gc[(12 * w + q) * kPThreads];
    const float2 mr[3] = {mul2(r, M[6]), mul2(r, M[7]), mul2(r, M[8])};  // r M^-1[2,:]
    float2 G[3][3], al1[3], al2[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float2 ax = A[w][c][0], ay = A[w][c][1], az = A[w][c][2];
#pragma unroll
      for (int x = 0; x < 3; ++x) G[c][x] = fma2(ax, M[x], fma2(ay, M[3 + x], mul2(az, mr[x])));
      if constexpr (HG) {
        // alpha_1 = (d_1 - a_zeta / 3) - k9 (2 a_xi - a_eta), alpha_2 = (d_2 - a_zeta / 3) - k9 (2 a_eta - a_xi)
        const float2 nk9 = p2(-lc.z, -lc.z), a3 = mul2(az, p2(1.f / 3.f, 1.f / 3.f));
        const float2 dl = sub2(ax, ay);
        al1[c] = fma2(nk9, add2(ax, dl), sub2(D1[HG ? w : 0][c], a3));
        al2[c] = fma2(nk9, sub2(ay, dl), sub2(D2[HG ? w : 0][c], a3));
      }
    }
    const float2 ve = mul2(mul2(vw2, gc[(12 * w + 9) * kPThreads]), eta[w]);
    const float2 ve2 = add2(ve, ve);
    float2 S[3][3];
    if (div_term) {
      const float2 vt = mul2(mul2(ve, p2(-2.f / 3.f, -2.f / 3.f)), add2(add2(G[0][0], G[1][1]), G[2][2]));
      S[0][0] = fma2(ve2, G[0][0], vt), S[1][1] = fma2(ve2, G[1][1], vt), S[2][2] = fma2(ve2, G[2][2], vt);
    } else {
      S[0][0] = mul2(ve2, G[0][0]), S[1][1] = mul2(ve2, G[1][1]), S[2][2] = mul2(ve2, G[2][2]);
    }
    S[0][1] = S[1][0] = mul2(ve, add2(G[0][1], G[1][0]));
    S[0][2] = S[2][0] = mul2(ve, add2(G[0][2], G[2][0]));
    S[1][2] = S[2][1] = mul2(ve, add2(G[1][2], G[2][1]));
    float2 nek = p2(0.f, 0.f), e3 = p2(0.f, 0.f);  // -eps k9, eps / 3
    if constexpr (HG) {
      const float2 eps = mul2(mul2(p2(hgk, hgk), eta[w]),
                              fma2(vw2, gc[(12 * w + 10) * kPThreads], mul2(p2(lc.w, lc.w), gc[(12 * w + 11) * kPThreads])));
      nek = mul2(eps, p2(-lc.z, -lc.z)), e3 = mul2(eps, p2(1.f / 3.f, 1.f / 3.f));
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float2 h0 = fma2(S[c][0], M[0], fma2(S[c][1], M[1], mul2(S[c][2], M[2])));
      float2 h1 = fma2(S[c][0], M[3], fma2(S[c][1], M[4], mul2(S[c][2], M[5])));
      const float2 h2 = fma2(S[c][0], mr[0], fma2(S[c][1], mr[1], mul2(S[c][2], mr[2])));
      if constexpr (HG) {
        // b_1 = 2 alpha_1 - alpha_2, b_2 = 2 alpha_2 - alpha_1 (b_1 + b_2 = alpha_1 + alpha_2)
        const float2 b1 = sub2(add2(al1[c], al1[c]), al2[c]), b2 = sub2(add2(al2[c], al2[c]), al1[c]);
        h0 = fma2(nek, b1, h0), h1 = fma2(nek, b2, h1);
        Y[w][0][c] = sub2(h2, mul2(e3, add2(al1[c], al2[c])));
        Y[w][HG ? 1 : 0][c] = fma2(e3, b1, h2), Y[w][HG ? 2 : 0][c] = fma2(e3, b2, h2);
      } else {
        Y[w][0][c] = h2;
      }
      H0[w][c] = h0, H1[w][c] = h1;
    }
  }
  // corners: 00 = W0 node 0, 11 = W1 node 0, 10 = W0 node 1 + W1 node 2, 01 = W0 node 2 + W1 node 1;
  // X = (-(h0 + h1), h0, h1) at a wedge's nodes (0, 1, 2); bottom X - Y, top X + Y
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float2 u0 = add2(H0[0][c], H1[0][c]), u3 = add2(H0[1][c], H1[1][c]);  // -X at 00 and 11
    const float2 x1 = add2(H0[0][c], H1[1][c]), x2 = add2(H1[0][c], H0[1][c]);
    float2 y0, y1, y2, y3;
    if constexpr (HG) {
      y0 = Y[0][0][c], y3 = Y[1][0][c];
      y1 = add2(Y[0][HG ? 1 : 0][c], Y[1][HG ? 2 : 0][c]), y2 = add2(Y[0][HG ? 2 : 0][c], Y[1][HG ? 1 : 0][c]);
    } else {
      y0 = Y[0][0][c], y3 = Y[1][0][c];
      y1 = y2 = add2(y0, y3);
    }
    bq[0][c] = add2(u0, y0), tq[0][c] = sub2(y0, u0);
    bq[3][c] = add2(u3, y3), tq[3][c] = sub2(y3, u3);
    bq[1][c] = sub2(x1, y1), tq[1][c] = add2(x1, y1);
    bq[2][c] = sub2(x2, y2), tq[2][c] = add2(x2, y2);
  }
}


// Ring buffer of the paired-cell tiles: one float4 (three components and a pad) per tile-line node,
// slot and layer, at ((slot n_r + k) 10 + d) RC + ring_index (slots as for the FP64 halo-free tiles:
// 2 bi + bj, bi = the node is on the tile's first row, bj = on its first column).
__device__ __forceinline__ int ring4_at(const RingDims& RD, int n_r, int slot, int k, int d, int rid) {
  return ((slot * n_r + k) * 10 + d) * RD.RC + rid;  // < 4 n_r 10 RC, far below 2^31 for N <= 256
}

// Levels with N >= 32 (tiles of 16 x 32 cells) whose three input arrays start on 16-byte
// boundaries; radial chunks of at most kPMaxKc cell layers.  FLAGS / EPI / EK as for k_tile.
template <bool HG, int FLAGS, int EPI, int EK>
__global__ void __launch_bounds__(kPThreads, 2)
    k_pair32(Dims D, OpA<float, HG> op, const float* __restrict__ in0, const float* __restrict__ in1,
             const float* __restrict__ in2, float* __restrict__ out0, float* __restrict__ out1,
             float* __restrict__ out2, const float* __restrict__ geo, const float* __restrict__ lay,
             EtaView<float> eta, const float* __restrict__ svec, int bc_in, int bc_out, int kc,
             const int* __restrict__ skip, EpiArgs<float> E, float4* __restrict__ ring) {
  extern __shared__ __align__(16) float psm[];
  float* const stg = psm;                                                   // [kPStages][kPStage]
  float* const exb = psm + kPStages * kPStage;                              // [2][3][kPExch]
  float2* const gc0 = reinterpret_cast<float2*>(exb + 2 * 3 * kPExch);      // [kPGeo][kPThreads]
  float4* const lct = reinterpret_cast<float4*>(gc0 + kPGeo * kPThreads);   // [kPMaxKc + 1]
  float2* const gc = gc0 + threadIdx.x;
  if (skip && *skip) return;
  const int N = D.N, n_r = D.n_r, P = D.P;
  const int LS = (int)D.layer_stride, NLL = (int)D.n_lat_layout;
  const int ntj = N / kPTJ;
  const int i0 = (blockIdx.x / ntj) * kPTI, j0 = (blockIdx.x % ntj) * kPTJ;
  const int d = blockIdx.z;
  const int kc0 = blockIdx.y * kc, kc1 = min(n_r - 1, kc0 + kc);
  const int kstart = kc0 > 0 ? kc0 - 1 : 0;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = i0 + 2 * w, j = j0 + lane;  // cell A = (i, j), cell B = (i + 1, j)
  const int dbase = (int)(d * D.diamond_stride);
  const int latb = d * (N + 1) * P;

  // Staging copies of this thread for layer L: node chunks h = 0, 1 (component c, node row
  // i0 + rr, nodes j0 + 4 q .. j0 + 4 q + 3 of node layer L; j0 + 35 <= N + 3 < P), and one chunk of
  // the viscosity of cell layer L (tile row rr, 16 bytes of the cells j0 .. j0 + 31).
  const float* srcn[2];
  uint32_t dstn[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int id = min((int)threadIdx.x + h * kPThreads, kPNodeChunks - 1);
    const int c = id / (kPRows * 9), rem = id % (kPRows * 9), rr = rem / 9, q = rem % 9;
    const float* base = c == 0 ? in0 : (c == 1 ? in1 : in2);
    srcn[h] = base + dbase + (i0 + rr) * P + j0 + 4 * q;
    dstn[h] = smem_u32(stg + (c * kPRows + rr) * kPRow + 4 * q);
  }
  const bool has1 = (int)threadIdx.x + kPThreads < kPNodeChunks;
  const char* srce;
  uint32_t dste;
  bool hase;
  {
    const int t = threadIdx.x;
    const int rows = ((d * (n_r - 1)) * N + i0) * N + j0;  // wedge pairs before the tile's first row
    if (EK == TN_ETA_F32) {  // 64 floats = 16 copies per row
      const int rr = t >> 4, q = t & 15;
      srce = reinterpret_cast<const char*>(eta.v + (rows + rr * N) * 2 + 4 * q);
      dste = smem_u32(stg + kPNodes + rr * 64 + 4 * q);
      hase = true;
    } else {  // 64 16-bit values = 8 copies per row
      const int rr = (t >> 3) & 15, q = t & 7;
      srce = reinterpret_cast<const char*>(eta.q + (rows + rr * N) * 2) + 16 * q;
      dste = smem_u32(stg + kPNodes) + rr * 128 + 16 * q;
      hase = t < 128;
    }
  }
  const int64_t eta_lb = (int64_t)N * N * 2 * (EK == TN_ETA_F32 ? 4 : 2);  // bytes per cell layer
  auto issue = [&](int L) {  // layer L into its buffer; one commit group per call
    if (L <= kc1) {
      const uint32_t so = (uint32_t)((L % kPStages) * kPStage * (int)sizeof(float));
      cp_async16(dstn[0] + so, srcn[0] + (int64_t)L * LS);
      if (has1) cp_async16(dstn[1] + so, srcn[1] + (int64_t)L * LS);
      if (L < kc1 && hase) cp_async16(dste + so, srce + L * eta_lb);
    }
    cp_async_commit();
  };
  // this thread's six nodes (i .. i + 2, j .. j + 1) at a staged node layer, as the corner pairs
  // (A, B) of corners 00, 10, 01, 11; projected on the boundary layers
  auto read_pairs = [&](int layer, float2 (&v)[4][3]) {
    const float* sg = stg + (layer % kPStages) * kPStage + (2 * w) * kPRow + lane;
    float n[6][3];  // node (i + a, j + b) at n[3 b + a]
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a) n[3 * b + a][c] = sg[c * kPRows * kPRow + a * kPRow + b];
    if ((FLAGS & PROJ_IN) && (layer == 0 || layer == n_r - 1)) {
      const int bc = layer == 0 ? bc_in : bc_out;
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a)
          project_vec(n[3 * b + a], svec, (int64_t)(latb + (i + a) * P + j + b), (int64_t)NLL, bc);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      v[0][c] = p2(n[0][c], n[1][c]), v[1][c] = p2(n[1][c], n[2][c]);
      v[2][c] = p2(n[3][c], n[4][c]), v[3][c] = p2(n[4][c], n[5][c]);
    }
  };
  // viscosity of the wedges (w0, w1) of cells A and B at cell layer k, from its staged layer
  auto read_eta = [&](int k, float2 (&e)[2]) {
    const float* se = stg + (k % kPStages) * kPStage + kPNodes;
    if (EK == TN_ETA_F32) {
      const float2 a = reinterpret_cast<const float2*>(se)[(2 * w) * 32 + lane];
      const float2 b = reinterpret_cast<const float2*>(se)[(2 * w + 1) * 32 + lane];
      e[0] = p2(a.x, b.x), e[1] = p2(a.y, b.y);
    } else {
      const uint32_t qa = reinterpret_cast<const uint32_t*>(se)[(2 * w) * 32 + lane];
      const uint32_t qb = reinterpret_cast<const uint32_t*>(se)[(2 * w + 1) * 32 + lane];
      e[0] = p2(from16<EK>((uint16_t)(qa & 0xffffu)), from16<EK>((uint16_t)(qb & 0xffffu)));
      e[1] = p2(from16<EK>((uint16_t)(qa >> 16)), from16<EK>((uint16_t)(qb >> 16)));
    }
  };

  // column values into shared memory, this CTA's layer constants into lct
  {
    const int nt = (int)D.n_tri;
    const int tA = ((d * N + i) * N + j) * 2, tB = tA + 2 * N;
#pragma unroll
    for (int wd = 0; wd < 2; ++wd) {
      float2 M[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) M[q] = gc[(12 * wd + q) * kPThreads] = p2(geo[q * nt + tA + wd], geo[q * nt + tB + wd]);
      float a = geo[9 * nt + tA + wd], b = geo[9 * nt + tB + wd];
      if (EK != TN_ETA_F32) a *= eta.cs[tA + wd], b *= eta.cs[tB + wd];
      const float2 dM = gc[(12 * wd + 9) * kPThreads] = p2(a, b);
      if constexpr (HG) {
        float2 l = p2(0.f, 0.f), qq = p2(0.f, 0.f);
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          const float2 s01 = add2(M[x], M[3 + x]);
          l = add2(l, add2(add2(mul2(s01, s01), mul2(M[x], M[x])), mul2(M[3 + x], M[3 + x])));
          qq = add2(qq, mul2(M[6 + x], M[6 + x]));
        }
        gc[(12 * wd + 10) * kPThreads] = mul2(mul2(p2(2.f, 2.f), dM), l);
        gc[(12 * wd + 11) * kPThreads] = mul2(mul2(p2(6.f, 6.f), dM), qq);
      }
    }
    for (int t = threadIdx.x; t < kc1 - kstart; t += kPThreads) {
      const float* l = lay + kLayerStride * (kstart + t);
      lct[t] = make_float4(l[4], l[5], l[8], l[9]);
    }
  }

  // outputs: nodes (i, j) and (i + 1, j) at on0 and on0 + P past the node layer's start; tile
  // lines to the ring (row lines at (i / 16) (N + 1) + j, column lines after RD.H)
  const RingDims RD = ring_dims(N, kPTI, kPTJ);
  const int on0 = dbase + i * P + j;
  const int rrow0 = (i0 / kPTI) * (N + 1) + j;                                  // node (i0, j)
  const int rcol0 = RD.H + (j0 / kPTJ) * (N - N / kPTI) + (i - i0 / kPTI - 1);  // node (i, j0) (i > i0)
  const int rcol1 = rcol0 + (N - N / kPTI);                                       // node (i, j0 + 32)
  const float lm = lane > 0 ? 1.f : 0.f;  // the left cells of column j0 belong to another tile
  auto store_node = [&](int k, int idx, float (&v)[3]) {  // a finished node inside the tile
    if ((FLAGS & PROJ_OUT) && (k == 0 || k == n_r - 1)) {
      const int bc = k == 0 ? bc_in : bc_out;
      const int64_t so = (int64_t)latb + (idx - dbase - k * LS);
      project_vec(v, svec, so, (int64_t)NLL, bc);
      if (FLAGS & ADD_ID) {
        float uu[3] = {in0[idx], in1[idx], in2[idx]};
        float pu[3] = {uu[0], uu[1], uu[2]};
        project_vec(pu, svec, so, (int64_t)NLL, bc);
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c] += uu[c] - pu[c];
      }
    }
    if (EPI != EPI_NONE) {
      epilogue<float, EPI>(E, in0, in1, in2, idx, v);
      return;
    }
    out0[idx] = v[0], out1[idx] = v[1], out2[idx] = v[2];
  };
  auto store4 = [&](int k, int idx, const float4& v4) {
    float v[3] = {v4.x, v4.y, v4.z};
    store_node(k, idx, v);
  };
  auto ring_put = [&](int k, int slot, int rid, const float4& v) { ring[ring4_at(RD, n_r, slot, k, d, rid)] = v; };
  // node layer kn from the corner totals of this thread's two cells (all radial contributions in):
  // sum the four cells around every node, store the nodes inside the tile, ring the tile lines
  auto finish_layer = [&](int kn, const float2 (&tot)[4][3]) {
    float* const ex = exb + (kn & 1) * 3 * kPExch;
    // node values as float4 (x, y, z = components, w unused): the ring takes them in one store
    float4 own0, own1, dn, r0, r1, r2;
    float* const o0 = &own0.x;
    float* const o1 = &own1.x;
    float* const on = &dn.x;
    float* const q0 = &r0.x;
    float* const q1 = &r1.x;
    float* const q2 = &r2.x;
    own0.w = own1.w = dn.w = r0.w = r1.w = r2.w = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float e0 = tot[0][c].x, e1 = tot[1][c].x + tot[0][c].y, e2 = tot[1][c].y;  // column j
      const float f0 = tot[2][c].x, f1 = tot[3][c].x + tot[2][c].y, f2 = tot[3][c].y;  // column j + 1
      const float F0 = __shfl_up_sync(0xffffffffu, f0, 1), F1 = __shfl_up_sync(0xffffffffu, f1, 1),
                  F2 = __shfl_up_sync(0xffffffffu, f2, 1);
      o0[c] = fmaf(F0, lm, e0), o1[c] = fmaf(F1, lm, e1), on[c] = fmaf(F2, lm, e2);
      q0[c] = f0, q1[c] = f1, q2[c] = f2;  // column j0 + 32 (lane 31)
      ex[c * kPExch + w * 33 + lane] = on[c];
      if (lane == 31) ex[c * kPExch + w * 33 + 32] = f2;
    }
    __syncthreads();
    if (w > 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        o0[c] += ex[c * kPExch + (w - 1) * 33 + lane];
        if (lane == 31) q0[c] += ex[c * kPExch + (w - 1) * 33 + 32];
      }
    }
    const int ok = on0 + kn * LS;
    if (lane > 0) {
      if (w > 0) store4(kn, ok, own0);
      store4(kn, ok + P, own1);
    } else {  // column j0
      if (w > 0) ring_put(kn, 1, rcol0, own0);
      ring_put(kn, 1, rcol0 + 1, own1);
    }
    if (w == 0) ring_put(kn, 2 + (lane == 0), rrow0, own0);                  // row i0
    if (w == 7) ring_put(kn, lane == 0, rrow0 + (N + 1), dn);                // row i0 + 16
    if (lane == 31) {                                                        // column j0 + 32
      if (w > 0) ring_put(kn, 0, rcol1, r0);
      else ring_put(kn, 2, rrow0 + 1, r0);
      ring_put(kn, 0, rcol1 + 1, r1);
      if (w == 7) ring_put(kn, 0, rrow0 + (N + 1) + 1, r2);
    }
  };
  // one cell layer: cin holds the top contributions of cell layer k - 1 to node layer k, cout
  // receives those of cell layer k to node layer k + 1
  auto step = [&](int k, const float2 (&cin)[4][3], float2 (&cout)[4][3]) {
    float2 tp[4][3], bt[4][3], e[2];
    read_pairs(k + 1, tp);
    read_pairs(k, bt);
    read_eta(k, e);
    // the buffer of layer k + kPAhead last held layer k - 1, read by every thread before the
    // previous barrier
    issue(k + kPAhead);
    float2 bq[4][3];
    pair_cell<HG>(tp, bt, gc, lct[k - kstart], e, op.div_term, op.hgk, bq, cout);
    cp_async_wait<kPAhead - 2>();  // layer k + 2 is in (made visible by the next barrier)
    if (k >= kc0) {
      float2 tot[4][3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        tot[0][c] = sub2(cin[0][c], bq[0][c]), tot[3][c] = sub2(cin[3][c], bq[3][c]);
        tot[1][c] = add2(cin[1][c], bq[1][c]), tot[2][c] = add2(cin[2][c], bq[2][c]);
      }
      finish_layer(k, tot);
    } else {
      __syncthreads();
    }
  };

#pragma unroll
  for (int q = 0; q < kPAhead; ++q) issue(kstart + q);
  cp_async_wait<kPAhead - 2>();  // layers kstart and kstart + 1 are in
  __syncthreads();               // ... for every thread, and so are lct and the column values
  float2 ca[4][3], cb[4][3];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int c = 0; c < 3; ++c) ca[q][c] = p2(0.f, 0.f);
  int k = kstart;
  for (; k + 1 < kc1; k += 2) {  // two layers per trip: the carried contributions swap arrays
    step(k, ca, cb);
    step(k + 1, cb, ca);
  }
  if (k < kc1) {
    step(k, ca, cb);
    if (kc1 == n_r - 1) finish_layer(n_r - 1, cb);
  } else if (kc1 == n_r - 1) {
    finish_layer(n_r - 1, ca);
  }
  cp_async_wait<0>();
}

// Sum of the ring partials of k_pair32 at tile-line node (i, j) of diamond d, node layer k: one
// partial per tile that has the node on its edge (slot 2 bi + bj; no tile beyond the diamond).
__device__ __forceinline__ void ring4_sum(const RingDims& RD, int N, int n_r, const float4* __restrict__ ring, int k,
                                          int d, int i, int j, float (&v)[3]) {
  const int rid = ring_index(RD, N, i, j);
  const bool on_h = i % RD.TI == 0, on_v = j % RD.TJ == 0;
  for (int bi = 0; bi < 2; ++bi) {
    if (bi == 1 && !on_h) break;
    if (on_h && ((bi == 0 && i == 0) || (bi == 1 && i == N))) continue;
    for (int bj = 0; bj < 2; ++bj) {
      if (bj == 1 && !on_v) break;
      if (on_v && ((bj == 0 && j == 0) || (bj == 1 && j == N))) continue;
      const float4 x = ring[ring4_at(RD, n_r, 2 * bi + bj, k, d, rid)];
      v[0] += x.x, v[1] += x.y, v[2] += x.z;
    }
  }
}

// Diamond-edge nodes of the paired-cell tiles, one thread per interface group g (the copies of one
// lattice point) and node layer k: the ring partials of every copy summed, the boundary rows
// projected and (I - P) u added once, then the value -- or the fused vector update -- at every
// copy (what k_ring_fix and k_interface do in two passes for the other tiles).
template <int EPI>
__global__ void k_ring4_edges(Dims D, RingDims RD, int n_groups, const int* __restrict__ gptr,
                              const int64_t* __restrict__ goff, const int4* __restrict__ gdij,
                              const float* __restrict__ gs, const float4* __restrict__ ring,
                              const float* __restrict__ in0, const float* __restrict__ in1,
                              const float* __restrict__ in2, float* __restrict__ out0, float* __restrict__ out1,
                              float* __restrict__ out2, int bc_in, int bc_out, const int* __restrict__ skip,
                              EpiArgs<float> E) {
  if (skip && *skip) return;
  const int g = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;  // grid: groups x layers
  if (g >= n_groups) return;
  const int N = D.N, n_r = D.n_r;
  const int b = gptr[g], e = gptr[g + 1];
  float v[3] = {0.f, 0.f, 0.f};
  for (int q = b; q < e; ++q) {
    const int4 c = gdij[q];
    ring4_sum(RD, N, n_r, ring, k, c.x, c.y, c.z, v);
  }
  const int lo = k * (int)D.layer_stride;
  if (k == 0 || k == n_r - 1) {
    const int bc = k == 0 ? bc_in : bc_out;
    const int o = (int)goff[b] + lo;
    const float w[3] = {in0[o], in1[o], in2[o]};
    if (bc == TN_BC_NOSLIP) {
      for (int c = 0; c < 3; ++c) v[c] = w[c];
    } else {
      const float s[3] = {gs[g], gs[n_groups + g], gs[2 * n_groups + g]};
      const float dv = v[0] * s[0] + v[1] * s[1] + v[2] * s[2], dw = w[0] * s[0] + w[1] * s[1] + w[2] * s[2];
      for (int c = 0; c < 3; ++c) v[c] += (dw - dv) * s[c];
    }
  }
  for (int q = b; q < e; ++q) {
    const int o = (int)goff[q] + lo;
    if (EPI != EPI_NONE) {
      epilogue<float, EPI>(E, in0, in1, in2, o, v);
    } else {
      out0[o] = v[0], out1[o] = v[1], out2[o] = v[2];
    }
  }
}

// Sums the ring partials of k_pair32 and finishes the tile-line nodes inside the diamond (as
// k_ring_fix does for the FP64 halo-free tiles); the diamond-edge nodes are k_ring4_edges'.
template <int FLAGS, int EPI>
__global__ void k_ring4_fix(Dims D, RingDims RD, const float4* __restrict__ ring, const float* __restrict__ in0,
                            const float* __restrict__ in1, const float* __restrict__ in2, float* __restrict__ out0,
                            float* __restrict__ out1, float* __restrict__ out2, const float* __restrict__ svec,
                            int bc_in, int bc_out, const int* __restrict__ skip, EpiArgs<float> E) {
  if (skip && *skip) return;
  const int N = D.N, n_r = D.n_r;
  const int rid = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y, d = blockIdx.z;  // grid: RC x n_r x 10
  if (rid >= RD.RC) return;
  int i, j;
  if (rid < RD.H) {
    i = (rid / (N + 1)) * RD.TI, j = rid % (N + 1);
  } else {
    const int r2 = rid - RD.H, per = N - N / RD.TI;
    const int t = r2 % per;
    j = (r2 / per) * RD.TJ;
    i = (t / (RD.TI - 1)) * RD.TI + 1 + t % (RD.TI - 1);
  }
  if (i == 0 || i == N || j == 0 || j == N) return;  // diamond edge
  float v[3] = {0.f, 0.f, 0.f};
  ring4_sum(RD, N, n_r, ring, k, d, i, j, v);
  const int M = N + 1;
  const int idx = (int)(d * D.diamond_stride) + k * (int)D.layer_stride + i * D.P + j;
  const int64_t so = ((int64_t)d * M + i) * D.P + j;
  if ((FLAGS & PROJ_OUT) && (k == 0 || k == n_r - 1)) {
    const int bc = k == 0 ? bc_in : bc_out;
    project_vec(v, svec, so, D.n_lat_layout, bc);
    if (FLAGS & ADD_ID) {
      float uu[3] = {in0[idx], in1[idx], in2[idx]};
      float pu[3] = {uu[0], uu[1], uu[2]};
      project_vec(pu, svec, so, D.n_lat_layout, bc);
      for (int c = 0; c < 3; ++c) v[c] += uu[c] - pu[c];
    }
  }
  if (EPI != EPI_NONE) {
    epilogue<float, EPI>(E, in0, in1, in2, idx, v);
    return;
  }
  out0[idx] = v[0], out1[idx] = v[1], out2[idx] = v[2];
}
