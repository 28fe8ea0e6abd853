// One Taylor-Horner step of exp(V) on the mixed-precision chain with the
// 5th-generation tensor cores: tcgen05.mma kind::tf32, 3xTF32 splitting
// (hi*hi + hi*lo + lo*hi, FP32 accumulation in TMEM), B operand streamed by
// TMA, A operand generated in shared memory from the walker's field table.
//
// Complex product as one real GEMM.  For 64 complex rows of the output the
// MMA rows are [Re C (64) ; Im C (64)] and the contraction index runs over
// [Re Z (Kp) ; Im Z (Kp)]:
//   Re C = Vr Zr - Vi Zi,   Im C = Vi Zr + Vr Zi,
// so the 128 x 2Kp A tile is [[Vr, -Vi], [Vi, Vr]] (rows of this walker's
// V gathered from phi) and the B tile is the chain stored K-major (row c =
// column c of Z as [Re | Im]), i.e. exactly the layout of the chain planes.
//
// Work item = one walker x one block of 64 complex rows x one column tile of
// NT <= 256 columns.  A persistent CTA walks a list of items; two
// shared-memory stages overlap the generation of A and the TMA of B for k
// tile t+1 with the MMAs of tile t (warp specialisation below).  Every
// mbarrier wait is bounded; on expiry the kernel sets bit 2 of the status
// word, drains its own copies and MMAs (bounded) and frees TMEM.
//
// Outputs the rows/columns covered by the MMA tile; k_chain_border handles
// the rest (for M = 257: row 256 and column 256).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "complex_math.cuh"
#include "ftq_internal.h"
#include "mixed_common.cuh"
#include "tc_common.cuh"

namespace ftq {
namespace {

using namespace tc;

constexpr int KTILE = 32;            // floats per k tile = 128 bytes = one swizzle row
constexpr int AROWS = 128;           // MMA M
constexpr long WAIT_LIMIT = TC_WAIT_LIMIT;


// Element (r, k) of a 128 x 32 K-major tile in the 128-byte swizzled layout
// sits at byte (r >> 3) * 1024 + (r & 7) * 128 + (((k >> 2) ^ (r & 7)) & 7) * 16
// + (k & 3) * 4; the generator below evaluates it incrementally.

struct TcArgs {
    const float* Yu;
    float* out;
    const float* Uf;              // the U term as one FP32 plane per walker
    float* Of;                    // nullable: the output also as one FP32 plane (last Horner step)
    const float2* phi;            // FP32 field table [W][nslot]
    const uint16_t* vidx;
    const float2* zs;             // scales as (hi, lo) float pairs, nullable
    const float2* us;
    const float2* os;
    const int* pk;                // packed basis coordinates [M]
    const uint16_t* qcube;        // difference -> slot [qsize]
    float alpha;
    int M, nslot, Kp, LDc, NT, ktiles;
    int qsize, qoff;
    int* status;
};

constexpr int MAXSYS = 8;
constexpr int NSMAX = 4;             // most k-tile stages the pipeline keeps in flight

// Up to MAXSYS systems in one launch: their chain tensor maps and arguments.
struct TcBatch {
    CUtensorMap maps[MAXSYS];
    TcArgs args[MAXSYS];
    int nsys;
    int nt_max;         // largest N tile over the systems (shared-memory layout)
    int nslot_max;
    int qsize_max;
    int m_max;
    int ncols;          // TMEM columns allocated once per CTA
    int nstage;         // shared-memory stages of the k-tile pipeline (2 .. NSMAX)
    long long wait_limit;   // polls per bounded mbarrier wait of the pipeline
};

// Persistent, warp-specialised kernel over a work list of items (system,
// walker, 64-row block, column tile), with the accumulator double-buffered in
// TMEM so that the epilogue of one item overlaps the MMAs of the next.
//   warps 0..3 (epilogue): wait until item i's accumulator (TMEM buffer i & 1)
//       is complete, read it lane quadrant by quadrant (warp w owns TMEM lanes
//       32w..32w+31), add the U term, split to tf32 hi + lo and store the
//       output planes; then release the buffer.
//   warps 4..11 (generators): build the A tile of every k tile into its
//       shared-memory stage and arrive on afull[stage].
//   warp 12, lane 0 (control): waits for A (afull), B (TMA) and, at the start
//       of an item, for its TMEM buffer to be released; issues the 12 MMAs of a
//       k tile, commits them to mma_bar[stage] (and after an item's last k tile
//       to tfull[buffer]); once the previous MMA group has drained it
//       prefetches the next B tile into the freed stage.
// Stage counters run over all k tiles of all items a CTA processes, buffer
// counters over its items, so mbarrier phases stay consistent.  An item with
// system index -1 ends the list (work lists compacted by the walkers' ranks
// keep their active items first); every role stops there.  Every wait is
// bounded; on expiry the kernel latches bit 2 of the status word, every role
// skips its remaining work (all warps still pass the same barriers), the
// control thread drains its own copies and MMAs, and TMEM is freed.
constexpr int NEPI = 128;                 // epilogue threads (4 warps)
constexpr int NGEN = 256;                 // generator threads (8 warps)
constexpr int NCTRL = 32;                 // control warp
constexpr int NTHREADS_WS = NEPI + NGEN + NCTRL;

__device__ __forceinline__ void gen_barrier() {
    asm volatile("bar.sync 1, %0;" ::"n"(NGEN) : "memory");
}

// Bounded wait that also gives up once another warp has latched an abort;
// the result is uniform over the calling warp's active lanes.
__device__ bool mbar_wait_ab(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* status,
                             long long limit) {
    bool ok = false;
    for (long long i = 0; i < limit && !ok; ++i) {
        if (*abort_flag) break;
        ok = mbar_try_wait(bar, parity);
    }
    ok = __all_sync(__activemask(), ok);
    if (!ok && !*abort_flag) {
        *abort_flag = 1;
        atomicOr(status, 2);
    }
    return ok;
}

__global__ void __launch_bounds__(NTHREADS_WS, 1) k_chain_tc(const __grid_constant__ TcBatch tb,
                                                             const int4* __restrict__ items, int nitems) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ uint64_t tma_bar[NSMAX], mma_bar[NSMAX], afull[NSMAX], tfull[2], tempty[2];
    __shared__ uint32_t tmem_sh;
    __shared__ volatile int abort_sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t pad = (1024u - (smem_u32(smem_raw) & 1023u)) & 1023u;
    unsigned char* base = smem_raw + pad;
    const uint32_t a_bytes = AROWS * KTILE * 4;
    const uint32_t bmax_bytes = (uint32_t)tb.nt_max * KTILE * 4;
    const uint32_t stage_bytes = 2 * a_bytes + 2 * bmax_bytes;
    const int NS = tb.nstage;
    float2* phs = reinterpret_cast<float2*>(base + (size_t)NS * stage_bytes);
    int* pks = reinterpret_cast<int*>(phs + tb.nslot_max);
    uint16_t* qs = reinterpret_cast<uint16_t*>(pks + tb.m_max);
    int* st = tb.args[0].status;

    if (tid == 0) {
        for (int b = 0; b < NSMAX; ++b) {
            mbar_init(&tma_bar[b], 1);
            mbar_init(&mma_bar[b], 1);
            mbar_init(&afull[b], NGEN / 32);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], NEPI / 32);
        }
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(&tmem_sh, 2u * (uint32_t)tb.ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_sh;

    if (warp == (NEPI + NGEN) / 32) {
        // ------------------------------------------------ control warp
        if (lane == 0) {
            int g = 0, last_mma = -1;
            int last_tma[NSMAX];
#pragma unroll
            for (int b = 0; b < NSMAX; ++b) last_tma[b] = -1;
            // prefetch cursor: the next k tile (over all items of this CTA)
            // whose B tile is to be loaded, and its global index pf_g
            int pf_item = blockIdx.x, pf_kt = 0, pf_g = 0;
            auto pf_valid = [&]() { return pf_item < nitems && items[pf_item].x >= 0; };
            auto prefetch = [&]() {
                const int4 it = items[pf_item];
                const TcArgs& q = tb.args[it.x];
                const int sg = pf_g % NS;
                unsigned char* Bh = base + sg * stage_bytes + 2 * a_bytes;
                mbar_expect_tx(&tma_bar[sg], 2u * (uint32_t)q.NT * KTILE * 4);
                tma_load_2d(Bh, &tb.maps[it.x], pf_kt * KTILE, (2 * it.y) * q.LDc + it.w * q.NT, &tma_bar[sg]);
                tma_load_2d(Bh + bmax_bytes, &tb.maps[it.x], pf_kt * KTILE, (2 * it.y + 1) * q.LDc + it.w * q.NT,
                            &tma_bar[sg]);
                last_tma[sg] = pf_g;
                ++pf_g;
                if (++pf_kt == q.ktiles) {
                    pf_kt = 0;
                    pf_item += gridDim.x;
                }
            };
            bool ok = true;
            while (pf_g < NS - 1 && pf_valid()) prefetch();      // NS - 1 tiles ahead
            int li = 0;                                   // items of this CTA so far
            for (int item = blockIdx.x; item < nitems && ok && items[item].x >= 0; item += gridDim.x, ++li) {
                const int4 it = items[item];
                const TcArgs& p = tb.args[it.x];
                const uint32_t idesc = idesc_tf32(p.NT);
                const int tb_i = li & 1;
                const uint32_t acc = tmem + (uint32_t)(tb_i * tb.ncols);
                // the epilogue of item li - 2 must have released this buffer
                if (li >= 2) ok = mbar_wait_ab(&tempty[tb_i], (uint32_t)(((li - 2) >> 1) & 1), &abort_sh, st, tb.wait_limit);
                for (int kt = 0; kt < p.ktiles && ok; ++kt, ++g) {
                    const int s = g % NS, use = g / NS;
                    ok = mbar_wait_ab(&afull[s], (uint32_t)(use & 1), &abort_sh, st, tb.wait_limit) &&
                         mbar_wait_ab(&tma_bar[s], (uint32_t)(use & 1), &abort_sh, st, tb.wait_limit);
                    if (!ok) break;
                    tc_fence_after();
                    unsigned char* Ahi = base + s * stage_bytes;
                    const uint64_t ah = sdesc_sw128(Ahi), al = sdesc_sw128(Ahi + a_bytes);
                    const uint64_t bh = sdesc_sw128(Ahi + 2 * a_bytes), bl = sdesc_sw128(Ahi + 2 * a_bytes + bmax_bytes);
#pragma unroll
                    for (int k = 0; k < KTILE / 8; ++k) {
                        const uint64_t dk = (uint64_t)((k * 32) >> 4);   // 8 tf32 = 32 bytes along the row
                        mma_tf32(acc, ah + dk, bh + dk, idesc, (kt > 0 || k > 0) ? 1u : 0u);
                        mma_tf32(acc, ah + dk, bl + dk, idesc, 1u);
                        mma_tf32(acc, al + dk, bh + dk, idesc, 1u);
                    }
                    mma_commit(&mma_bar[s]);
                    if (kt + 1 == p.ktiles) mma_commit(&tfull[tb_i]);   // accumulator complete
                    last_mma = g;
                    // the next B tile goes into the stage of tile pf_g - NS
                    // (= g - 1 in steady state), once its MMAs are done
                    if (pf_valid()) {
                        if (pf_g >= NS)
                            ok = mbar_wait_ab(&mma_bar[pf_g % NS], (uint32_t)(((pf_g - NS) / NS) & 1), &abort_sh, st,
                                              tb.wait_limit);
                        if (!ok) break;
                        prefetch();
                    }
                }
            }
            if (!ok) {   // abort latched: drain this CTA's own copies and MMAs
                for (int b = 0; b < NS; ++b)
                    if (last_tma[b] >= 0) mbar_wait(&tma_bar[b], (uint32_t)((last_tma[b] / NS) & 1));
                if (last_mma >= 0) mbar_wait(&mma_bar[last_mma % NS], (uint32_t)((last_mma / NS) & 1));
            }
        }
    } else if (warp >= NEPI / 32) {
        // ------------------------------------------------ generator warps
        // Loop bounds are uniform over these warps, so after an abort they
        // still pass the same named barriers; only the work is skipped.
        const int gw = warp - NEPI / 32, gt = tid - NEPI;
        int g = 0;
        int loaded_sys = -1;
        // swizzled offsets: row j = gw + 8 t has (j & 7) = gw and (j >> 3) = t
        const uint32_t off_top = (uint32_t)(gw * 128 + ((((lane >> 2) ^ gw) & 7) << 4) + (lane & 3) * 4);
        for (int item = blockIdx.x; item < nitems && items[item].x >= 0; item += gridDim.x) {
            const int4 it = items[item];
            const TcArgs& p = tb.args[it.x];
            const int w = it.y, rows0 = it.z * 64;
            const float2* ph = p.phi + (long)w * p.nslot;
            gen_barrier();        // every generator is done with the previous item's tables
            for (int i = gt; i < p.nslot; i += NGEN) phs[i] = ph[i];
            if (it.x != loaded_sys) {
                for (int i = gt; i < p.M; i += NGEN) pks[i] = p.pk[i];
                for (int i = gt; i < p.qsize; i += NGEN) qs[i] = p.qcube[i];
                loaded_sys = it.x;
            }
            gen_barrier();
            int prow[64 / (NGEN / 32)];
#pragma unroll
            for (int t = 0; t < 64 / (NGEN / 32); ++t) {
                const int i = rows0 + gw + t * (NGEN / 32);
                prow[t] = i < p.M ? pks[i] + p.qoff : -1;
            }
            for (int kt = 0; kt < p.ktiles; ++kt, ++g) {
                const int s = g % NS, use = g / NS;
                if (g >= NS && !mbar_wait_ab(&mma_bar[s], (uint32_t)((use - 1) & 1), &abort_sh, st, tb.wait_limit)) continue;
                if (abort_sh) continue;
                unsigned char* Ahi = base + s * stage_bytes;
                unsigned char* Alo = Ahi + a_bytes;
                const int kg = kt * KTILE + lane;
                const bool im_half = kg >= p.Kp;
                const int kc = im_half ? kg - p.Kp : kg;
                const ScaleF zsc((p.zs != nullptr && kc < p.M) ? p.zs[kc] : make_float2(1.f, 0.f));
                const int pkc = kc < p.M ? pks[kc] : 0;
#pragma unroll
                for (int t = 0; t < 64 / (NGEN / 32); ++t) {
                    float2 v = make_float2(0.f, 0.f);
                    if (prow[t] >= 0 && kc < p.M) {
                        v = phs[qs[prow[t] - pkc]];        // V[i][k] = phi(n_i - n_k)
                        v.x = zsc(v.x);
                        v.y = zsc(v.y);
                    }
                    const float top = im_half ? -v.y : v.x;
                    const float bot = im_half ? v.x : v.y;
                    float h, l;
                    split_tf32(top, h, l);
                    uint32_t o = off_top + (uint32_t)t * 1024u;          // element (gw + 8 t, lane)
                    *reinterpret_cast<float*>(Ahi + o) = h;
                    *reinterpret_cast<float*>(Alo + o) = l;
                    split_tf32(bot, h, l);
                    o += 8u * 1024u;                                     // row 64 + j
                    *reinterpret_cast<float*>(Ahi + o) = h;
                    *reinterpret_cast<float*>(Alo + o) = l;
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&afull[s]);
            }
        }
    } else {
        // ------------------------------------------------ epilogue warps
        int li = 0;
        for (int item = blockIdx.x; item < nitems && items[item].x >= 0; item += gridDim.x, ++li) {
            const int4 it = items[item];
            const TcArgs& p = tb.args[it.x];
            const int tb_i = li & 1;
            const bool acc_ok = mbar_wait_ab(&tfull[tb_i], (uint32_t)((li >> 1) & 1), &abort_sh, st, tb.wait_limit);
            tc_fence_after();
            const int w = it.y, rows0 = it.z * 64, col0 = it.w * p.NT;
            const int r = warp * 32 + lane;               // accumulator row = TMEM lane
            const int i = rows0 + (r & 63);
            const int part = r >> 6;                      // 0: Re C, 1: Im C
            const bool row_ok = i < p.M;
            const ScaleF usi(row_ok ? p.us[i] : make_float2(0.f, 0.f));
            const ScaleF osi((row_ok && p.os != nullptr) ? p.os[i] : make_float2(1.f, 0.f));
            const size_t rowlen = 2 * (size_t)p.Kp;
            const size_t partoff = (size_t)p.LDc * rowlen;
            const size_t wstride = 2 * partoff;
            const float* __restrict__ U = p.Uf + partoff * w;      // one plane per walker
            float* __restrict__ O = p.out + wstride * w;
            float* __restrict__ Of = p.Of ? p.Of + partoff * w : nullptr;
            const int cend = min(col0 + p.NT, p.M);
            const uint32_t acc = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(tb_i * tb.ncols);
            const int nch = (p.NT + 15) / 16;
            // U of chunk ch + 1 is loaded while chunk ch is finished, so that two
            // chunks of loads are in flight per thread; U is read as one FP32
            // plane (it equals hi + lo of the chain planes exactly)
            float uf[3][16];
            auto load_u = [&](int ch, float (&u)[16]) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int c = col0 + ch * 16 + q;
                    const size_t o = (size_t)c * rowlen + (size_t)part * p.Kp + i;
                    u[q] = (row_ok && c < cend) ? U[o] : 0.f;
                }
            };
            auto finish = [&](int ch, const uint32_t (&v)[16], const float (&u)[16]) {
                if (!row_ok) return;
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int c = col0 + ch * 16 + q;
                    if (c < cend) {
                        const size_t o = (size_t)c * rowlen + (size_t)part * p.Kp + i;
                        const float val = osi(fmaf(p.alpha, __uint_as_float(v[q]), usi(u[q])));
                        float hh, ll;
                        split_tf32(val, hh, ll);
                        O[o] = hh;
                        O[partoff + o] = ll;
                        if (Of) Of[o] = val;
                    }
                }
            };
            if (acc_ok) {
#pragma unroll
                for (int d = 0; d < 3 - 1; ++d)
                    if (d < nch) load_u(d, uf[d]);
                for (int ch0 = 0; ch0 < nch; ch0 += 3) {
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const int ch = ch0 + d;
                        if (ch < nch) {
                            if (ch + 3 - 1 < nch) load_u(ch + 3 - 1, uf[(d + 3 - 1) % 3]);
                            uint32_t v[16];
                            tmem_ld16(acc + (uint32_t)(ch * 16), v);
                            finish(ch, v, uf[d]);
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[tb_i]);    // this warp's quadrant is read
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 2u * (uint32_t)tb.ncols);
}

// Output entries outside the MMA tile: rows [R, M) x all columns and
// columns [NT, M) x rows [0, R), on CUDA cores in FP32 from the same
// hi + lo operands.  A border row of V (or a border column of Z) is staged in
// shared memory once and reused for every output of that row (column).
__device__ __forceinline__ void border_store(float* O, const float* U, const Planes& P, const double* us,
                                             const double* os, float alpha, int i, int c, float2 acc) {
    float2 u = P.load(U, i, c);
    const ScaleF s(us[i]);
    float2 val = make_float2(fmaf(alpha, acc.x, s(u.x)), fmaf(alpha, acc.y, s(u.y)));
    if (os) {
        const ScaleF o(os[i]);
        val.x = o(val.x);
        val.y = o(val.y);
    }
    P.store(O, i, c, val);
}

__device__ __forceinline__ float2 warp_sum(float2 v) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// One warp per output entry, lanes over the contraction index (coalesced
// reads of the chain rows), V from the shared difference cube.  Eight blocks
// per SM (at most 32 registers) keep 1024 walkers in one wave, and two
// partial sums per lane keep eight chain loads in flight.
__global__ void __launch_bounds__(256, 8) k_chain_border(const float* __restrict__ Zin, const float* __restrict__ Yu,
                                                     float* __restrict__ out, const double2* __restrict__ phi,
                                                     const int* __restrict__ pk, const uint16_t* __restrict__ qcube,
                                                     const double* __restrict__ zs, const double* __restrict__ us,
                                                     const double* __restrict__ os, float alpha, int M, int nslot,
                                                     int qsize, int qoff, Planes P, size_t wstride, int R, int NT) {
    extern __shared__ unsigned char smem_raw[];
    float2* vec = reinterpret_cast<float2*>(smem_raw);     // [M]: one row of V zs or one column of Z zs
    float2* phs = vec + M;                                  // [nslot]
    int* pks = reinterpret_cast<int*>(phs + nslot);         // [M]
    uint16_t* qs = reinterpret_cast<uint16_t*>(pks + M);    // [qsize]
    const int w = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const float* Z = Zin + wstride * w;
    const float* U = Yu + wstride * w;
    float* O = out + wstride * w;
    const double2* ph = phi + (long)w * nslot;
    const int Rr = R < M ? R : M;
    for (int e = threadIdx.x; e < nslot; e += blockDim.x) {
        const double2 d = ph[e];
        phs[e] = make_float2((float)d.x, (float)d.y);
    }
    for (int e = threadIdx.x; e < M; e += blockDim.x) pks[e] = pk[e];
    for (int e = threadIdx.x; e < qsize; e += blockDim.x) qs[e] = qcube[e];
    __syncthreads();
    for (int i = Rr; i < M; ++i) {              // border rows: (V zs)[i, :] Z
        for (int k = threadIdx.x; k < M; k += blockDim.x) {
            const ScaleF sk(zs ? zs[k] : 1.0);
            const float2 v = phs[qs[pks[i] - pks[k] + qoff]];
            vec[k] = make_float2(sk(v.x), sk(v.y));
        }
        __syncthreads();
        for (int c = warp; c < M; c += nw) {
            float2 acc = make_float2(0.f, 0.f), acc2 = make_float2(0.f, 0.f);
            int k = lane;
            for (; k + 32 < M; k += 64) {
                const float2 z0 = P.load(Z, k, c), z1 = P.load(Z, k + 32, c);
                acc = cfma(vec[k], z0, acc);
                acc2 = cfma(vec[k + 32], z1, acc2);
            }
            if (k < M) acc = cfma(vec[k], P.load(Z, k, c), acc);
            acc = warp_sum(acc + acc2);
            if (lane == 0) border_store(O, U, P, us, os, alpha, i, c, acc);
        }
        __syncthreads();
    }
    for (int c = NT; c < M; ++c) {              // border columns: (V zs)[:R, :] Z[:, c]
        for (int k = threadIdx.x; k < M; k += blockDim.x) {
            const ScaleF sk(zs ? zs[k] : 1.0);
            const float2 z = P.load(Z, k, c);
            vec[k] = make_float2(sk(z.x), sk(z.y));
        }
        __syncthreads();
        for (int i = warp; i < Rr; i += nw) {
            const int base = pks[i] + qoff;
            float2 acc = make_float2(0.f, 0.f);
            for (int k = lane; k < M; k += 32) acc = cfma(phs[qs[base - pks[k]]], vec[k], acc);
            acc = warp_sum(acc);
            if (lane == 0) border_store(O, U, P, us, os, alpha, i, c, acc);
        }
        __syncthreads();
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }
    return fn;
}

}  // namespace

// Tile plan for basis size M with nct column tiles: rows covered by 64-row
// MMA blocks (R, possibly padded above M) and the MMA N width (<= 256).
void tc_plan(int M, int nct, int* R, int* NT) {
    int rem = M % 64;
    if (rem == 0) *R = M;
    else if (M > 64 && rem <= 8) *R = M - rem;          // a thin border row band on CUDA cores
    else *R = (M + 63) / 64 * 64;                       // padded rows, not stored
    if (M <= 256 * nct) *NT = ((M + nct - 1) / nct + 15) / 16 * 16;
    else *NT = 256;                                     // border columns [256 nct, M) on CUDA cores
}

// Dynamic shared memory of k_chain_tc: nstage stages of A (hi, lo) and B
// (hi, lo) tiles, the field table, the packed basis and the difference cube.
size_t tc_smem_bytes(int nt_max, int nslot_max, int m_max, int qsize_max, int nstage) {
    const size_t stage = 2 * (size_t)AROWS * KTILE * 4 + 2 * (size_t)nt_max * KTILE * 4;
    return 1024 + (size_t)nstage * stage + sizeof(float2) * nslot_max + sizeof(int) * m_max +
           sizeof(uint16_t) * qsize_max;
}

constexpr size_t TC_SMEM_LIMIT = 227 * 1024 - 2048;   // leaves room for the kernel's static shared memory

// The deepest pipeline (2 .. NSMAX stages) whose shared memory fits; 0 when
// not even two stages do.  More stages keep more B tiles in flight, which
// hides the TMA latency behind the MMAs of the tiles before.
int tc_stages(int nt_max, int nslot_max, int m_max, int qsize_max) {
    for (int ns = NSMAX; ns >= 2; --ns)
        if (tc_smem_bytes(nt_max, nslot_max, m_max, qsize_max, ns) <= TC_SMEM_LIMIT) return ns;
    return 0;
}

bool tc_fits(const ftq_ctx* c, int nct) {
    int R, NT;
    tc_plan(c->M, nct, &R, &NT);
    const int qsize = c->sys.qS * c->sys.qS * c->sys.qS;
    return tc_stages(NT, c->nslot, c->M, qsize) >= 2;
}

// The fewest column tiles (1 .. 8) whose tile width lets the shared memory
// fit; 0 when none does.
int tc_min_nct(const ftq_ctx* c) {
    for (int nct = 1; nct <= 8; ++nct)
        if (tc_fits(c, nct)) return nct;
    return 0;
}

bool tc_supported(int M) {
    (void)M;
    return encode_fn() != nullptr;
}

int tmem_cols(int NT) { return NT <= 32 ? 32 : (NT <= 64 ? 64 : (NT <= 128 ? 128 : 256)); }

// One tensor map per chain buffer: [W * 2 * LDc rows] x [2 Kp floats],
// boxes of 32 floats x NT rows, 128-byte swizzle; and the work list.
cudaError_t tc_make_maps(ftq_ctx* c) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const int nmin = tc_min_nct(c);
    if (nmin == 0) return cudaErrorInvalidValue;
    if (c->nct < nmin) c->nct = nmin;
    int R, NT;
    tc_plan(c->M, c->nct, &R, &NT);
    float* bufs[3] = {c->Ypl, c->zpl[0], c->zpl[1]};
    for (int b = 0; b < 3; ++b) {
        cuuint64_t dims[2] = {(cuuint64_t)(2 * c->Kp), (cuuint64_t)c->W * 2 * c->LD};
        cuuint64_t strides[1] = {(cuuint64_t)(2 * c->Kp) * sizeof(float)};
        cuuint32_t box[2] = {(cuuint32_t)KTILE, (cuuint32_t)NT};
        cuuint32_t estr[2] = {1, 1};
        CUtensorMap* m = reinterpret_cast<CUtensorMap*>(c->tmap[b]);
        CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, bufs[b], dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
        c->tmap_buf[b] = bufs[b];
    }
    std::vector<int4> items;
    for (int w = 0; w < c->W; ++w)
        for (int rb = 0; rb < R / 64; ++rb)
            for (int ct = 0; ct < c->nct; ++ct) items.push_back(make_int4(0, w, rb, ct));
    if (c->items) cudaFree(c->items);
    c->items = nullptr;
    if (c->items_lr) cudaFree(c->items_lr);      // rebuilt from the ranks at the next stabilisation
    c->items_lr = nullptr;
    cudaError_t e = cudaMalloc(&c->items, sizeof(int4) * items.size());
    if (e != cudaSuccess) return e;
    c->nitems = (int)items.size();
    return cudaMemcpy(c->items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice);
}

namespace {

bool fill_args(ftq_ctx* c, const float* zin, float* out, const double* zs, const double* os, float alpha,
               TcArgs* a, CUtensorMap* map, int* NTo) {
    const CUtensorMap* m = nullptr;
    for (int b = 0; b < 3; ++b)
        if (c->tmap_buf[b] == zin) m = reinterpret_cast<const CUtensorMap*>(c->tmap[b]);
    if (!m) return false;
    *map = *m;
    int R, NT;
    tc_plan(c->M, c->nct, &R, &NT);
    a->Yu = c->Ypl;
    a->out = out;
    a->Uf = c->Yf;
    a->Of = os ? c->Yf : nullptr;         // the last Horner step's output becomes the new Y
    a->phi = c->phi32;
    a->vidx = c->tab.vidx;
    a->zs = zs ? c->tab.hf : nullptr;     // the only scale the chain uses is h
    a->us = c->tab.hf;
    a->os = os ? c->tab.hf : nullptr;
    a->pk = c->tab.pk;
    a->qcube = c->tab.qcube;
    a->qsize = c->sys.qS * c->sys.qS * c->sys.qS;
    a->qoff = c->sys.qoff;
    a->alpha = alpha;
    a->M = c->M;
    a->nslot = c->nslot;
    a->Kp = c->Kp;
    a->LDc = c->LD;
    a->NT = NT;
    a->ktiles = 2 * c->Kp / KTILE;
    a->status = c->status;
    *NTo = NT;
    return true;
}

cudaError_t launch_items(ftq_ctx* timing_ctx, TcBatch& tb, const int4* items, int nitems, cudaStream_t st) {
    tb.nstage = tc_stages(tb.nt_max, tb.nslot_max, tb.m_max, tb.qsize_max);
    if (tb.nstage < 2) return cudaErrorInvalidValue;
    const size_t smem = tc_smem_bytes(tb.nt_max, tb.nslot_max, tb.m_max, tb.qsize_max, tb.nstage);
    static size_t smem_set = 0;
    cudaError_t e = cudaSuccess;
    if (smem > smem_set) {
        e = cudaFuncSetAttribute(k_chain_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        smem_set = smem;
    }
    int dev = 0, sms = 0, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_chain_tc, NTHREADS_WS, smem);
    per_sm = std::min(per_sm, 512 / (2 * tb.ncols));   // two accumulators per CTA in 512 TMEM columns
    if (per_sm < 1) per_sm = 1;
    const int grid = std::min(nitems, sms * per_sm);
    LaunchScope ls(timing_ctx, FTQ_K_CHAIN);
    k_chain_tc<<<grid, NTHREADS_WS, smem, st>>>(tb, items, nitems);
    return cudaGetLastError();
}

cudaError_t launch_border(ftq_ctx* c, const float* zin, float* out, const double* zs, const double* os, float alpha) {
    int R, NT;
    tc_plan(c->M, c->nct, &R, &NT);
    if (R >= c->M && NT * c->nct >= c->M) return cudaSuccess;
    Planes P;
    P.Kp = c->Kp;
    P.part = (size_t)c->LD * 2 * c->Kp;
    const int qsize = c->sys.qS * c->sys.qS * c->sys.qS;
    const size_t bsm = sizeof(float2) * (c->M + c->nslot) + sizeof(int) * c->M + sizeof(uint16_t) * qsize;
    static size_t bsm_set = 48 * 1024;
    if (bsm > bsm_set) {
        cudaError_t e = cudaFuncSetAttribute(k_chain_border, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsm);
        if (e != cudaSuccess) return e;
        bsm_set = bsm;
    }
    LaunchScope ls(c, FTQ_K_BORDER);
    k_chain_border<<<c->W, 256, bsm, c->stream>>>(zin, c->Ypl, out, c->phi, c->tab.pk, c->tab.qcube, zs, c->tab.h, os,
                                                 alpha, c->M, c->nslot, qsize, c->sys.qoff, P, 2 * P.part, R,
                                                 NT * c->nct);
    return cudaGetLastError();
}

}  // namespace

cudaError_t tc_chain_step(ftq_ctx* c, const float* zin, float* out, const double* zs, const double* os,
                          float alpha) {
    TcBatch tb;
    std::memset(&tb, 0, sizeof(tb));
    int NT;
    if (!fill_args(c, zin, out, zs, os, alpha, &tb.args[0], &tb.maps[0], &NT)) return cudaErrorInvalidValue;
    tb.nsys = 1;
    tb.nt_max = NT;
    tb.nslot_max = c->nslot;
    tb.m_max = c->M;
    tb.qsize_max = tb.args[0].qsize;
    tb.ncols = tmem_cols(NT);
    tb.wait_limit = c->wait_limit >= 0 ? (long long)c->wait_limit : (long long)WAIT_LIMIT;
    const int4* items = (c->opts.low_rank_threshold > 0.0 && c->items_lr) ? c->items_lr : c->items;
    cudaError_t e = launch_items(c, tb, items, c->nitems, c->stream);
    if (e != cudaSuccess) return e;
    return launch_border(c, zin, out, zs, os, alpha);
}

// One Horner step for every member of a batch in one persistent launch.
cudaError_t tc_chain_step_batch(ftq_ctx* b, const float* const* zin, float* const* out, int j, int p) {
    TcBatch tb;
    std::memset(&tb, 0, sizeof(tb));
    const int ns = (int)b->members.size();
    if (ns > MAXSYS) return cudaErrorInvalidValue;
    tb.nsys = ns;
    for (int s = 0; s < ns; ++s) {
        ftq_ctx* c = b->members[s];
        int NT;
        if (!fill_args(c, zin[s], out[s], j == p ? c->tab.h : nullptr, j == 1 ? c->tab.h : nullptr, 1.0f / j,
                       &tb.args[s], &tb.maps[s], &NT))
            return cudaErrorInvalidValue;
        tb.nt_max = std::max(tb.nt_max, NT);
        tb.nslot_max = std::max(tb.nslot_max, c->nslot);
        tb.m_max = std::max(tb.m_max, c->M);
        tb.qsize_max = std::max(tb.qsize_max, tb.args[s].qsize);
        tb.ncols = std::max(tb.ncols, tmem_cols(NT));
    }
    tb.wait_limit = b->wait_limit >= 0 ? (long long)b->wait_limit : (long long)WAIT_LIMIT;
    cudaError_t e = launch_items(b, tb, b->items, b->nitems, b->stream);
    for (int s = 0; s < ns && e == cudaSuccess; ++s) {
        ftq_ctx* c = b->members[s];
        e = launch_border(c, zin[s], out[s], j == p ? c->tab.h : nullptr, j == 1 ? c->tab.h : nullptr, 1.0f / j);
    }
    return e;
}

namespace {

// Work list of a low-rank context: the items whose column tile starts below
// the walker's rank (ws[12]), in the order of the full list, then -1 entries.
__global__ void k_items_by_rank(const int4* __restrict__ all, int n, const double* __restrict__ ws, int NT,
                                int4* __restrict__ out) {
    __shared__ int base;
    __shared__ int cnt[1024];
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) base = 0;
    __syncthreads();
    for (int c0 = 0; c0 < n; c0 += nt) {
        const int i = c0 + tid;
        int keep = 0;
        int4 it = make_int4(-1, 0, 0, 0);
        if (i < n) {
            it = all[i];
            keep = (double)(it.w * NT) < ws[(long)WSTRIDE * it.y + 12] ? 1 : 0;
        }
        cnt[tid] = keep;
        __syncthreads();
        // inclusive scan of the chunk's flags (Hillis-Steele)
        for (int o = 1; o < nt; o <<= 1) {
            const int v = tid >= o ? cnt[tid - o] : 0;
            __syncthreads();
            cnt[tid] += v;
            __syncthreads();
        }
        if (keep) out[base + cnt[tid] - 1] = it;
        __syncthreads();
        if (tid == nt - 1) base += cnt[tid];
        __syncthreads();
    }
    for (int i = base + tid; i < n; i += nt) out[i] = make_int4(-1, 0, 0, 0);
}

}  // namespace

cudaError_t tc_items_by_rank(ftq_ctx* c) {
    if (!c->items_lr) {
        cudaError_t e = cudaMalloc(&c->items_lr, sizeof(int4) * (size_t)c->nitems);
        if (e != cudaSuccess) return e;
    }
    int R, NT;
    tc_plan(c->M, c->nct, &R, &NT);
    k_items_by_rank<<<1, 1024, 0, c->stream>>>(c->items, c->nitems, c->wstate, NT, c->items_lr);
    return cudaGetLastError();
}

// Work list of a batch: every member's items, largest basis first.
cudaError_t tc_batch_items(ftq_ctx* b) {
    std::vector<int> order(b->members.size());
    for (size_t s = 0; s < order.size(); ++s) order[s] = (int)s;
    std::sort(order.begin(), order.end(), [&](int x, int y) { return b->members[x]->M > b->members[y]->M; });
    std::vector<int4> items;
    for (int s : order) {
        ftq_ctx* c = b->members[s];
        int R, NT;
        tc_plan(c->M, c->nct, &R, &NT);
        for (int w = 0; w < c->W; ++w)
            for (int rb = 0; rb < R / 64; ++rb)
                for (int ct = 0; ct < c->nct; ++ct) items.push_back(make_int4(s, w, rb, ct));
    }
    if (b->items) cudaFree(b->items);
    b->items = nullptr;
    cudaError_t e = cudaMalloc(&b->items, sizeof(int4) * items.size());
    if (e != cudaSuccess) return e;
    b->nitems = (int)items.size();
    return cudaMemcpy(b->items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice);
}

// Time one Horner step (scratch output) for each column-tile count and keep
// the fastest; returns the chosen count.
cudaError_t tc_autotune(ftq_ctx* c, int* best_nct, float* best_ms) {
    int best = c->nct;
    float bms = 1e30f;
    const int n0 = tc_min_nct(c) > 0 ? tc_min_nct(c) : 1;
    const int cands[3] = {n0, n0 + 1, n0 + 2};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaError_t e = cudaSuccess;
    for (int nct : cands) {
        int R, NT;
        tc_plan(c->M, nct, &R, &NT);
        if (nct > 1 && NT * (nct - 1) >= c->M) continue;   // an empty column tile
        if (!tc_fits(c, nct)) continue;
        c->nct = nct;
        e = tc_make_maps(c);
        if (e != cudaSuccess) break;
        e = tc_chain_step(c, c->Ypl, c->zpl[0], nullptr, nullptr, 1.0f);   // warm-up
        if (e != cudaSuccess) break;
        cudaEventRecord(e0, c->stream);
        for (int r = 0; r < 3; ++r) tc_chain_step(c, c->Ypl, c->zpl[0], nullptr, nullptr, 1.0f);
        cudaEventRecord(e1, c->stream);
        e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= 3.f;
        if (ms < bms) { bms = ms; best = nct; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    c->nct = best;
    *best_nct = best;
    *best_ms = bms;
    return tc_make_maps(c);
}

}  // namespace ftq
