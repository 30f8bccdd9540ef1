// dct2d_pipe_kernels.cuh - persistent, software-pipelined four-step passes.
//
// The same arithmetic as dct2d_fs_kernels.cuh (four-step column FFTs, the
// radix-64 row pass with the fused split / postprocess / preprocess of
// Algorithm 2 and Section III), restructured so that memory and compute
// overlap inside every SM:
//
//  * one persistent CTA per SM, 256 threads = two consumer groups of 128;
//  * a ring of three shared-memory buffers; the input of an item (1 KB row
//    segments of a column slab, or four 16 KB rows of a row pass) is fetched
//    by the TMA engine (cp.async.bulk) with completion on an mbarrier, three
//    items ahead of the compute;
//  * each group computes its item in place in its buffer (named barrier per
//    group), the column steps write the result back with bulk stores, and the
//    freed buffer immediately receives the load of the item three ahead.
//
// Every mbarrier wait is bounded; a wait that gives up sets the plan's device
// error word, the CTA drains its own outstanding copies (again bounded) and
// returns.
#pragma once

#include "dct2d_fs_kernels.cuh"
#include "pipe.cuh"

namespace gbdct {

constexpr int kPipeBuf = 3;
constexpr int kPipeGroup = 128;
constexpr int kPipeThreads = 2 * kPipeGroup;

// ----------------------------------------------------------------------------
// Column steps of the four-step column FFT (N1 = A * B).
//   KIND 0: forward C1  (item: n1a, column block)  B input rows -> B workspace rows
//   KIND 1: forward C2  (item: k1b, column block)  A rows in place
//   KIND 2: inverse C2' (item: k1b, column block)  A rows in place
//   KIND 3: inverse C1' (item: n1a, column block)  B workspace rows -> B output rows
// ----------------------------------------------------------------------------
template <int N1, int KIND>
struct FsColOp {
  using G = FsGeom<N1>;
  static constexpr bool INV = KIND >= 2;
  static constexpr int NR = (KIND == 0 || KIND == 3) ? G::B : G::A;
  static constexpr int SET = (KIND == 0 || KIND == 3) ? G::A : G::B;
  static constexpr size_t BUF_BYTES = (size_t)G::ROWS * kFsCols * sizeof(float2);
  static constexpr int LOAD_SEGS = NR;
  static constexpr int STORE_SEGS = NR;
  static constexpr uint32_t SEG_BYTES = kFsCols * sizeof(float2);
  static constexpr uint32_t LOAD_BYTES = NR * SEG_BYTES;

  __device__ static int nitems(const Dct2dArgs& a, int batch) { return SET * (a.n2 / 2 / kFsCols) * batch; }
  __device__ static void decode(const Dct2dArgs& a, int item, int& r, int& cb, int& bz) {
    const int ncb = a.n2 / 2 / kFsCols;
    r = item % SET;
    cb = (item / SET) % ncb;
    bz = item / (SET * ncb);
  }
  // workspace row holding slab row i of this item
  __device__ static int work_row(int r, int i) {
    return (KIND == 1 || KIND == 2) ? r * G::A + i : i * G::A + r;
  }
  __device__ static const void* load_src(const Dct2dArgs& a, int item, int i) {
    int r, cb, bz;
    decode(a, item, r, cb, bz);
    if constexpr (KIND == 0) {
      return a.in + (long long)bz * a.in_bstride + (long long)reorder_src(r + G::A * i, N1) * a.n2 + cb * 2 * kFsCols;
    } else {
      return a.work + (long long)bz * a.work_bstride + (long long)work_row(r, i) * (a.n2 / 2) + cb * kFsCols;
    }
  }
  __device__ static void* store_dst(const Dct2dArgs& a, int item, int i) {
    int r, cb, bz;
    decode(a, item, r, cb, bz);
    if constexpr (KIND == 3) {
      return a.out + (long long)bz * a.out_bstride + (long long)reorder_src(r + G::A * i, N1) * a.n2 + cb * 2 * kFsCols;
    } else {
      return a.work + (long long)bz * a.work_bstride + (long long)work_row(r, i) * (a.n2 / 2) + cb * kFsCols;
    }
  }
  __device__ static uint32_t load_off(int i) { return i * SEG_BYTES; }
  __device__ static uint32_t load_bytes(int) { return SEG_BYTES; }

  template <int BAR>
  __device__ static void compute(const Dct2dArgs& a, int item, unsigned char* buf, int c) {
    float2* st = reinterpret_cast<float2*>(buf);
    int r, cb, bz;
    decode(a, item, r, cb, bz);
    float2 v[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) v[j] = st[j * kFsCols + c];
    r64::dft<NR, INV>(v);
    if constexpr (KIND == 0) {
#pragma unroll
      for (int k = 1; k < NR; ++k) v[k] = cmul(v[k], __ldg(a.fstw + r * G::B + k));
    } else if constexpr (KIND == 2) {
#pragma unroll
      for (int n = 1; n < NR; ++n) v[n] = cmulc(v[n], __ldg(a.fstw + n * G::B + r));
    }
#pragma unroll
    for (int k = 0; k < NR; ++k) st[k * kFsCols + c] = v[k];
  }
};

// ----------------------------------------------------------------------------
// Row passes (L = N2 = 4096): forward (split + row FFT + postprocess) and
// inverse (preprocess + row IFFT + column pairing).  Item b = rows k1 = 2b,
// 2b+1 (two sequences); the four input rows are staged by bulk copies.
// ----------------------------------------------------------------------------
template <int N1, int L, bool INV>
struct FsRowOp {
  using R = R64Geom<L>;
  static constexpr uint32_t ROW_BYTES = INV ? L * sizeof(float) : (L / 2) * sizeof(float2);
  static constexpr size_t BUF_BYTES = (4 * (size_t)ROW_BYTES > R::SMEM) ? 4 * (size_t)ROW_BYTES : R::SMEM;
  static constexpr int LOAD_SEGS = 4;
  static constexpr int STORE_SEGS = 0;
  static constexpr uint32_t LOAD_BYTES = 4 * ROW_BYTES;
  static_assert(R::THREADS == kPipeGroup, "one item per consumer group");

  __device__ static int nitems(const Dct2dArgs&, int batch) { return (N1 / 4) * batch; }
  __device__ static int mirror(int k1) { return k1 == 0 ? N1 / 2 : N1 - k1; }
  __device__ static const void* load_src(const Dct2dArgs& a, int item, int i) {
    const int b = item % (N1 / 4), bz = item / (N1 / 4);
    const int k1 = 2 * b + (i >> 1);
    const int row = (i & 1) ? mirror(k1) : k1;
    if constexpr (INV) {
      return a.in + (long long)bz * a.in_bstride + (long long)row * L;
    } else {
      return a.work + (long long)bz * a.work_bstride + (long long)fs_prow<N1>(row) * (L / 2);
    }
  }
  __device__ static void* store_dst(const Dct2dArgs&, int, int) { return nullptr; }
  __device__ static uint32_t load_off(int i) { return i * ROW_BYTES; }
  __device__ static uint32_t load_bytes(int) { return ROW_BYTES; }

  template <int BAR>
  __device__ static void compute(const Dct2dArgs& a, int item, unsigned char* sbuf, int gt) {
    const int s = gt & 1, t = gt >> 1;
    const int b = item % (N1 / 4), bz = item / (N1 / 4);
    const int k1 = 2 * b + s;
    const bool packed = (k1 == 0);
    const int kmir = mirror(k1);
    float2 v[r64::PMAX];
    if constexpr (!INV) {
      const float2* za_row = reinterpret_cast<const float2*>(sbuf + (2 * s) * ROW_BYTES);
      const float2* zb_row = reinterpret_cast<const float2*>(sbuf + (2 * s + 1) * ROW_BYTES);
#pragma unroll
      for (int j = 0; j < R::R1; ++j) {
        const int n2 = t + j * R::ST1;
        const bool lowhalf = n2 < L / 2;
        const int p = lowhalf ? n2 : L - 1 - n2;
        const float2 za = za_row[p];
        const float2 zb = zb_row[p];
        if (packed) {
          v[j] = lowhalf ? make_float2(za.x, zb.x) : make_float2(za.y, zb.y);
        } else {
          v[j] = lowhalf ? make_float2(0.5f * (za.x + zb.x), 0.5f * (za.y - zb.y))
                         : make_float2(0.5f * (za.y + zb.y), 0.5f * (zb.x - za.x));
        }
      }
    } else {
      const float* ca = reinterpret_cast<const float*>(sbuf + (2 * s) * ROW_BYTES);
      const float* cb = reinterpret_cast<const float*>(sbuf + (2 * s + 1) * ROW_BYTES);
      const float2 ia = __ldg(a.ia + k1);
      const float2 ih = __ldg(a.ia + N1 / 2);
#pragma unroll
      for (int j = 0; j < R::R1; ++j) {
        const int k2 = t + j * R::ST1;
        const int km = (L - k2) & (L - 1);
        const float c1 = ca[k2], c3 = cb[k2];
        const float c4 = k2 ? ca[km] : 0.f;
        const float c2 = k2 ? cb[km] : 0.f;
        const float2 bk = __ldg(a.ib + k2);
        if (packed) {
          const float2 v0 = cmul(cmul(make_float2(c1, -c4), bk), ia);
          const float2 vh = cmul(cmul(make_float2(c3 - c2, -(c3 + c2)), bk), ih);
          v[j] = make_float2(v0.x - vh.y, v0.y + vh.x);
        } else {
          v[j] = cmul(cmul(make_float2(c1 - c2, -(c3 + c4)), bk), ia);
        }
      }
    }
    pipe::named_sync<BAR, kPipeGroup>();  // staged rows consumed; the FFT reuses the buffer
    float2* buf = reinterpret_cast<float2*>(sbuf) + s * R::LP;
    r64::first_stage<L, INV>(v, buf, t);
    pipe::named_sync<BAR, kPipeGroup>();
    r64::stages_to_regs<L, R::R1, INV, BAR, kPipeGroup>(buf, t, a.tw2, v);
#pragma unroll
    for (int qb = 0; qb < R::NBL; ++qb)
#pragma unroll
      for (int m = 0; m < R::RL; ++m) buf[r64::pidx(r64::out_pos<L>(t, qb, m))] = v[qb * R::RL + m];
    pipe::named_sync<BAR, kPipeGroup>();

    if constexpr (!INV) {
      float* y = a.out + (long long)bz * a.out_bstride;
      const float2 av = __ldg(a.fa + k1);
      float* row0 = y + (long long)k1 * L;
      float* row1 = y + (long long)kmir * L;
      constexpr float RH = 0.70710678118654752f;
      for (int i = t; i < L / 8; i += R::TPS) {
        const int c = 4 * i;
        float2 Yq[5], Ym[5];
#pragma unroll
        for (int d = 0; d < 5; ++d) {
          Yq[d] = buf[r64::pidx(c + d)];
          Ym[d] = buf[r64::pidx((L - c - d) & (L - 1))];
        }
        float q0[4], q1[4], r0[4], r1[4];
#pragma unroll
        for (int d = 1; d <= 3; ++d) {
          const float2 bt = __ldg(a.fb + c + d);
          const float2 P = Yq[d], M = Ym[d];
          if (packed) {
            const float2 s0 = cmul(bt, make_float2(P.x + M.x, P.y - M.y));
            const float2 sh = cmul(bt, make_float2(RH * (P.y + M.y), RH * (M.x - P.x)));
            q0[d] = s0.x;
            q1[d] = sh.x;
            r0[4 - d] = -s0.y;
            r1[4 - d] = -sh.y;
          } else {
            const float2 aP = cmul(P, av);
            const float2 aM = cmul(M, av);
            const float2 sv = cmul(bt, make_float2(aP.x + aM.x, aP.y - aM.y));
            const float2 tv = cmul(bt, make_float2(aP.x - aM.x, aP.y + aM.y));
            q0[d] = sv.x;
            q1[d] = -tv.y;
            r0[4 - d] = -sv.y;
            r1[4 - d] = -tv.x;
          }
        }
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int col = e ? (L - c - 4) : c;
          const float2 P = e ? Ym[4] : Yq[0];
          const float2 M = e ? Yq[4] : Ym[0];
          const float2 bt = __ldg(a.fb + col);
          float o0, o1;
          if (packed) {
            const float2 s0 = cmul(bt, make_float2(P.x + M.x, P.y - M.y));
            const float2 sh = cmul(bt, make_float2(RH * (P.y + M.y), RH * (M.x - P.x)));
            o0 = s0.x;
            o1 = sh.x;
          } else {
            const float2 aP = cmul(P, av);
            const float2 aM = cmul(M, av);
            const float2 u = make_float2(aP.x + aM.x, aP.y - aM.y);
            const float2 w = make_float2(aP.x - aM.x, aP.y + aM.y);
            o0 = bt.x * u.x - bt.y * u.y;
            o1 = -(bt.x * w.y + bt.y * w.x);
          }
          if (e) { r0[0] = o0; r1[0] = o1; } else { q0[0] = o0; q1[0] = o1; }
        }
        *reinterpret_cast<float4*>(row0 + c) = make_float4(q0[0], q0[1], q0[2], q0[3]);
        *reinterpret_cast<float4*>(row1 + c) = make_float4(q1[0], q1[1], q1[2], q1[3]);
        *reinterpret_cast<float4*>(row0 + L - c - 4) = make_float4(r0[0], r0[1], r0[2], r0[3]);
        *reinterpret_cast<float4*>(row1 + L - c - 4) = make_float4(r1[0], r1[1], r1[2], r1[3]);
      }
    } else {
      float2* Zw = a.work + (long long)bz * a.work_bstride;
      float2* zr0 = Zw + (long long)fs_prow<N1>(k1) * (L / 2);
      float2* zr1 = Zw + (long long)fs_prow<N1>(kmir) * (L / 2);
      for (int p = t; p < L / 2; p += R::TPS) {
        const float2 u = buf[r64::pidx(p)];
        const float2 w = buf[r64::pidx(L - 1 - p)];
        if (packed) {
          zr0[p] = make_float2(u.x, w.x);
          zr1[p] = make_float2(u.y, w.y);
        } else {
          zr0[p] = make_float2(u.x - w.y, u.y + w.x);
          zr1[p] = make_float2(u.x + w.y, w.x - u.y);
        }
      }
    }
  }
};

// ----------------------------------------------------------------------------
// The persistent pipeline
// ----------------------------------------------------------------------------
template <class Op>
__host__ __device__ constexpr size_t pipe_smem_bytes() {
  return kPipeBuf * Op::BUF_BYTES + 64;  // buffers + mbarriers + issue counters
}

// bar.red.or over the 128 threads of consumer group `grp` (named barrier 1 + grp).
__device__ __forceinline__ bool group_any(bool pred, int grp) {
  int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.s32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, %3, p;\n\t"
      "selp.s32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((int)pred), "r"(1 + grp), "n"(kPipeGroup)
      : "memory");
  return r != 0;
}

template <class Op>
__global__ void __launch_bounds__(kPipeThreads, 1) k_pipe(Dct2dArgs a, int batch) {
  extern __shared__ __align__(128) unsigned char psm[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(psm + kPipeBuf * Op::BUF_BYTES);
  int* issued = reinterpret_cast<int*>(bars + kPipeBuf);  // loads issued per buffer
  const int grp = threadIdx.x / kPipeGroup, gt = threadIdx.x % kPipeGroup;
  const int lane = threadIdx.x & 31;
  const bool issuer = gt < 32;  // first warp of each group issues copies
  const int nitems = Op::nitems(a, batch);
  const int nk = (int)blockIdx.x < nitems ? (nitems - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

  if (threadIdx.x == 0) {
    for (int b = 0; b < kPipeBuf; ++b) {
      pipe::mbar_init(&bars[b], 1);
      issued[b] = 0;
    }
    pipe::fence_mbar_init();
  }
  __syncthreads();

  auto issue_load = [&](int k) {  // one full warp
    const int item = blockIdx.x + k * gridDim.x;
    const int b = k % kPipeBuf;
    unsigned char* buf = psm + b * Op::BUF_BYTES;
    if (lane == 0) {
      issued[b] += 1;
      pipe::mbar_arrive_expect_tx(&bars[b], Op::LOAD_BYTES);
    }
    __syncwarp();
    for (int i = lane; i < Op::LOAD_SEGS; i += 32)
      pipe::bulk_load(buf + Op::load_off(i), Op::load_src(a, item, i), Op::load_bytes(i), &bars[b]);
  };

  if (threadIdx.x < 32) {
    for (int k = 0; k < kPipeBuf && k < nk; ++k) issue_load(k);
  }

  for (int k = grp; k < nk; k += 2) {
    const int item = blockIdx.x + k * gridDim.x;
    const int b = k % kPipeBuf;
    unsigned char* buf = psm + b * Op::BUF_BYTES;
    const bool ok = pipe::mbar_wait(&bars[b], (k / kPipeBuf) & 1);
    if (group_any(!ok, grp)) {
      if (gt == 0) atomicExch(a.err, 1);
      break;
    }
    if (grp == 0) Op::template compute<1>(a, item, buf, gt);
    else Op::template compute<2>(a, item, buf, gt);
    if constexpr (Op::STORE_SEGS > 0) pipe::fence_proxy_async();
    if (grp == 0) pipe::named_sync<1, kPipeGroup>();
    else pipe::named_sync<2, kPipeGroup>();
    if (issuer) {
      if constexpr (Op::STORE_SEGS > 0) {
        for (int i = lane; i < Op::STORE_SEGS; i += 32)
          pipe::bulk_store(Op::store_dst(a, item, i), buf + Op::load_off(i), Op::load_bytes(i));
        pipe::bulk_commit();
        pipe::bulk_wait_read_all();
      }
      __syncwarp();
      if (k + kPipeBuf < nk) {
        pipe::fence_proxy_async();
        issue_load(k + kPipeBuf);
      }
    }
  }

  if (issuer) pipe::bulk_wait_all();
  __syncthreads();
  // Drain: every load issued into a buffer must have landed before the CTA
  // exits (normally already true; bounded after an error).
  if (threadIdx.x == 0) {
    for (int b = 0; b < kPipeBuf; ++b) {
      if (issued[b] > 0 && !pipe::mbar_wait(&bars[b], (issued[b] - 1) & 1)) atomicExch(a.err, 1);
    }
  }
}

}  // namespace gbdct
