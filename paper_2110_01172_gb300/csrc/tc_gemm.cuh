// tc_gemm.cuh - split-BF16 DFT-GEMM on the 5th-generation tensor cores
// (tcgen05.mma, operands staged by TMA, FP32 accumulator in tensor memory).
//
// One CTA computes one 128 x BN tile of D = A B^T for row-major ("K-major")
// operands A (rows x K) and B (cols x K), each given as a bf16 pair hi + lo:
//   D = Ah Bh^T + Ah Bl^T + Al Bh^T
// (the lo lo term is dropped), all three products accumulated into the same
// FP32 accumulator in tensor memory.  K advances in blocks of 64 elements: the
// four operand tiles of a block (128 x 64 and BN x 64 bf16, 128-byte rows with
// the 128-byte swizzle) arrive by tiled tensor loads into a ring of NST
// shared-memory stages; one thread issues the loads and the MMAs (K = 16 per
// instruction) and releases a stage with tcgen05.commit when the MMAs that
// read it are done.  The four warps then read the accumulator rows back with
// tcgen05.ld (warp w owns lanes 32w .. 32w+31, lane = tile row) and apply the
// epilogue:
//   EPI_SPLIT_T   row r of the tile is (batch b, n1) = (r / N1, r % N1) of the
//                 first product T = x M^T; it is stored transposed and split,
//                 Th/Tl[b][col][n1], as the K-major operand of the second
//                 product
//   EPI_F32       row r is output row k1 of batch entry blockIdx.z; stored as
//                 FP32, out[b][k1][col]
// Every mbarrier wait is bounded (poll limit); a wait that gives up records
// the failure in the device error word, the issuing thread stops issuing,
// waits (with the default limit) for the copies it issued and commits, so the
// epilogue and the tensor-memory release happen only after all issued work has
// completed; the tile is then left unwritten.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tma_util.cuh"

namespace gbdct {
namespace tc {

constexpr int BM = 128;                  // tile rows (MMA M)
constexpr int BK = 64;                   // K per stage: one 128-byte swizzle row of bf16
constexpr uint32_t kDefaultPolls = tma::kDefaultPolls;
using tma::bar_wait;
using tma::su32;
enum { EPI_SPLIT_T = 0, EPI_F32 = 1 };

template <int BN>
struct Cfg {
  static constexpr int A_BYTES = BM * BK * 2;             // 16 KB
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;  // hi + lo of both operands
  static constexpr int NST = BN >= 128 ? 3 : 4;
  static constexpr int SMEM = NST * STAGE + 1024 /* alignment */ + 256 /* barriers, TMEM slot */;
  // kind::f16 instruction descriptor: D f32, A and B bf16, both K-major, N, M
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                    ((uint32_t)(BM >> 4) << 24);
};

struct Epi {
  int mode;                 // EPI_SPLIT_T or EPI_F32
  int n1, n2;               // transform sides
  int a_batch_rows;         // A row offset per blockIdx.z
  int b_batch_rows;         // B row offset per blockIdx.z
  __nv_bfloat16* th;        // EPI_SPLIT_T outputs
  __nv_bfloat16* tl;
  float* out;               // EPI_F32 output
};

// Shared-memory matrix descriptor of a K-major bf16 tile with the 128-byte
// swizzle: 8-row groups of 128-byte rows, 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(const void* p) {
  const uint64_t a = su32(p);
  return ((a >> 4) & 0x3FFFull) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

__device__ __forceinline__ void tma_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(su32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(su32(bar))
      : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}

template <int BN>
__global__ void __launch_bounds__(128, 1)
k_tc_dftgemm(const __grid_constant__ CUtensorMap mah, const __grid_constant__ CUtensorMap mal,
             const __grid_constant__ CUtensorMap mbh, const __grid_constant__ CUtensorMap mbl, Epi e, int kblocks,
             uint32_t polls, int* err) {
  using C = Cfg<BN>;
  constexpr int NST = C::NST;
  extern __shared__ __align__(1024) unsigned char tc_raw[];
  unsigned char* sm = tc_raw + ((1024 - (su32(tc_raw) & 1023)) & 1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + NST * C::STAGE);
  uint64_t* empty = full + NST;
  uint64_t* done = empty + NST;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  int* fail = reinterpret_cast<int*>(tslot + 1);
  const int warp = threadIdx.x / 32;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int arow = e.a_batch_rows * (int)blockIdx.z + m0;
  const int brow = e.b_batch_rows * (int)blockIdx.z + n0;

  if (threadIdx.x == 0) {
    for (int i = 0; i < NST; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(full + i)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(empty + i)) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(done)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *fail = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)), "r"(BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  if (threadIdx.x == 0) {
    auto stage_ptr = [&](int s) { return sm + s * C::STAGE; };
    auto load = [&](int kb) {
      unsigned char* st = stage_ptr(kb % NST);
      uint64_t* fb = full + (kb % NST);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(fb)), "r"((uint32_t)C::STAGE)
                   : "memory");
      const int k = kb * BK;
      tma_2d(st, &mah, k, arow, fb);
      tma_2d(st + C::A_BYTES, &mal, k, arow, fb);
      tma_2d(st + 2 * C::A_BYTES, &mbh, k, brow, fb);
      tma_2d(st + 2 * C::A_BYTES + C::B_BYTES, &mbl, k, brow, fb);
    };
    int issued = 0, consumed = 0;
    bool ok = true;
    for (; issued < NST && issued < kblocks; ++issued) load(issued);
    for (int kb = 0; kb < kblocks && ok; ++kb) {
      const int s = kb % NST;
      if (!bar_wait(full + s, (kb / NST) & 1, polls)) {
        ok = false;
        break;
      }
      consumed = kb + 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      unsigned char* st = stage_ptr(s);
      unsigned char* ah = st;
      unsigned char* al = st + C::A_BYTES;
      unsigned char* bh = st + 2 * C::A_BYTES;
      unsigned char* bl = bh + C::B_BYTES;
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        const int off = kk * 32;  // 16 bf16 along the swizzled 128-byte row
        const uint32_t first = (kb == 0 && kk == 0) ? 0u : 1u;
        mma_bf16(tmem, sw128_desc(ah + off), sw128_desc(bh + off), C::IDESC, first);
        mma_bf16(tmem, sw128_desc(ah + off), sw128_desc(bl + off), C::IDESC, 1u);
        mma_bf16(tmem, sw128_desc(al + off), sw128_desc(bh + off), C::IDESC, 1u);
      }
      commit(empty + s);
      // refill the stage of block kb-1 once its MMAs are done
      if (kb >= 1 && issued < kblocks) {
        const int ps = (kb - 1) % NST;
        if (!bar_wait(empty + ps, ((kb - 1) / NST) & 1, polls)) {
          ok = false;
          break;
        }
        load(issued++);
      }
    }
    if (!ok) {
      *fail = 1;
      atomicExch(err, 1);
      // copies issued but not consumed must land before the CTA exits
      for (int kb = consumed; kb < issued; ++kb) bar_wait(full + kb % NST, (kb / NST) & 1, kDefaultPolls);
    }
    commit(done);  // arrives once every MMA issued so far has completed
  }
  __syncwarp();
  const bool fin = bar_wait(done, 0, kDefaultPolls);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (!fin && threadIdx.x == 0) atomicExch(err, 1);
  if (fin && !*fail) {
    const int r = warp * 32 + (threadIdx.x & 31);  // tile row = TMEM lane
    const int row = m0 + r;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
      uint32_t v[16];
      const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(ta));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (e.mode == EPI_F32) {
        float* o = e.out + ((long long)blockIdx.z * e.n1 + row) * e.n2 + n0 + c0;
#pragma unroll
        for (int i = 0; i < 16; i += 4)
          *reinterpret_cast<float4*>(o + i) = make_float4(__uint_as_float(v[i]), __uint_as_float(v[i + 1]),
                                                          __uint_as_float(v[i + 2]), __uint_as_float(v[i + 3]));
      } else {
        const int b = row / e.n1, n1 = row % e.n1;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const float x = __uint_as_float(v[i]);
          const __nv_bfloat16 h = __float2bfloat16_rn(x);
          const long long idx = ((long long)b * e.n2 + n0 + c0 + i) * e.n1 + n1;
          e.th[idx] = h;
          e.tl[idx] = __float2bfloat16_rn(x - __bfloat162float(h));
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
}

}  // namespace tc
}  // namespace gbdct
