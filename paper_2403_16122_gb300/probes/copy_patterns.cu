// copy_patterns.cu -- copy-only ceilings of the memory access patterns the
// step kernels use, on a 1024 x 1024 lattice (no physics: every variant reads
// what a step reads, in the order and granularity it reads it, and writes what
// a step writes; a few FMAs keep the data live). Standalone: not part of the
// library; its measurements back the choice of the blocked state layout.
//   v0  planar layout, per-lane cp.async gathers (the staged strip kernel's
//       pattern), per-lane stores; optional paired stores (v0p)
//   v1  planar layout, one bulk copy (cp.async.bulk on an mbarrier) per plane
//       segment and pull row, per-lane stores; optional paired stores (v1p)
//   v3  blocked layout (all planes of a 32-site block together), one bulk copy
//       per source row block, per-lane stores into the block
//   v4  blocked layout, one bulk copy per plane of a pull row (24 per row)
//   v5  blocked layout with the planes grouped by the row they stream from:
//       three chunk copies (rows y - 1, y, y + 1) and the own-site block per
//       pull row -- the pattern of the block step kernel
// FP32 (256 B per lattice update) and 16-bit (176 B) sizes; padding columns
// and rows keep every halo access in bounds. Build and run on the GPU:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 -o copy_patterns copy_patterns.cu
//   ./copy_patterns <measured copy GB/s> [variant filter] [rows per item] [repetitions]
#include <cstdio>
#include <cstdlib>
#include <cstdint>
#include <vector>
#include <cstring>
#include <algorithm>
#include <cuda_runtime.h>
#include <cuda_fp16.h>

#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { printf("CUDA %s at %d: %s\n", #x, __LINE__, cudaGetErrorString(e_)); exit(1);} } while (0)

constexpr int NX = 1024, NY = 1024, PADX = 32;
constexpr int PITCH = NX + 2 * PADX;    // 1088
constexpr int NYP = NY + 4;  // two padding rows on each side
constexpr long long PLANE = (long long)PITCH * NYP;  // 1116288
__host__ __device__ constexpr int CX(int i) { return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0); }
__host__ __device__ constexpr int CY(int i) { return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0); }
__device__ __forceinline__ long long site_of(int x, int y) { return (long long)(y + 2) * PITCH + PADX + x; }

struct Item { int x0, y0, y1, pad; };

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cpa(void* dst, const void* src, int n) {
    if (n == 16) asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
    else if (n == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void mbar_init(uint64_t* m, unsigned cnt) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(cnt) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t* m, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* m, unsigned parity) {
    unsigned ok;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(ok) : "r"(smem_u32(m)), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* m) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(m)) : "memory");
}
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, unsigned bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// bounded wait; false after the limit (the caller raises the error word)
__device__ __forceinline__ bool mbar_wait(uint64_t* m, unsigned parity) {
    for (int k = 0; k < (1 << 22); ++k)
        if (mbar_try(m, parity)) return true;
    return false;
}

// ---------------------------------------------------------------- layouts
// ST = float (FP32) or unsigned short (FP16). Population region: (g_i,h_i) pairs
// at 2(i-1)plane + 2site, f_i at (15+i)plane + site. aux (float): own0 4site,
// own1 4plane + 4site, FP16 only ref 8plane + 2site.
template <typename ST> struct L;
template <> struct L<float> {
    static constexpr int kGH = 36, kGH0 = 2;   // gh segment sites, start offset (x0 - kGH0)
    static constexpr int kF = 40, kF0 = 4;
    static constexpr int kNseg = 18;
    static constexpr int kGHb = kGH * 8, kFb = kF * 4, kOwnb = 36 * 16, kRefb = 0;
    static constexpr int kSlot = 8 * kGHb + 8 * kFb + 2 * kOwnb;  // 4736
    static constexpr int kOut = 8 * 256 + 8 * 128 + 2 * 512;      // 4096
};
template <> struct L<unsigned short> {
    static constexpr int kGH = 40, kGH0 = 4;
    static constexpr int kF = 48, kF0 = 8;
    static constexpr int kNseg = 19;
    static constexpr int kGHb = kGH * 4, kFb = kF * 2, kOwnb = 36 * 16, kRefb = 36 * 8;
    static constexpr int kSlot = 8 * kGHb + 8 * kFb + 2 * kOwnb + kRefb;  // 3488
    static constexpr int kOut = 8 * 128 + 8 * 64 + 2 * 512 + 256;           // 2816
};

struct Bufs { void* pop; float* aux; };

// ---------------------------------------------------------------- V0
template <typename ST, int STG, bool PAIR>
__global__ void __launch_bounds__(128, 2) v0(Bufs in, Bufs out, const Item* items, int n_items) {
    constexpr bool H = sizeof(ST) == 2;
    constexpr int SLOTF = H ? 34 * 32 : 32 * 32;  // floats per slot
    extern __shared__ __align__(16) float sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int it = blockIdx.x * 4 + warp;
    if (it >= n_items) return;
    const Item W = items[it];
    float* ring = sm + warp * STG * SLOTF;
    const int xc = W.x0 - 1 + lane;
    const bool outl = lane >= 1 && lane <= 30 && xc < NX;
    const float* A = (const float*)in.pop;
    const unsigned short* A16 = (const unsigned short*)in.pop;
    const int R = W.y1 - W.y0 + 2;
    auto issue = [&](int j) {
        if (j < R) {
            float* s = ring + (j % STG) * SLOTF;
            const int y = W.y0 - 1 + j;
            const long long own = site_of(xc, y);
            cpa(s + 4 * lane, in.aux + 4 * own, 16);
            cpa(s + 128 + 4 * lane, in.aux + 4 * PLANE + 4 * own, 16);
            if (H) cpa(s + 1024 + 2 * lane, in.aux + 8 * PLANE + 2 * own, 8);
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                const long long src = site_of(xc - CX(i), y - CY(i));
                if (H) {
                    cpa(s + 256 + 64 * (i - 1) + 2 * lane, A16 + 2 * (i - 1) * PLANE + 2 * src, 4);
                    cpa(s + 768 + 32 * (i - 1) + lane, A16 + (((15 + i) * PLANE + src) & ~1LL), 4);
                } else {
                    cpa(s + 256 + 64 * (i - 1) + 2 * lane, A + 2 * (i - 1) * PLANE + 2 * src, 8);
                    cpa(s + 768 + 32 * (i - 1) + lane, A + (15 + i) * PLANE + src, 4);
                }
            }
        }
        cpa_commit();
    };
#pragma unroll
    for (int j = 0; j < STG; ++j) issue(j);
    cpa_wait<STG - 2>();  // rows 0 and 1 landed (as the step kernel)
    for (int y = W.y0; y < W.y1; ++y) {
        const int jy = y - W.y0 + 1;
        issue(jy + STG - 1);
        cpa_wait<STG - 2>();  // row jy + 1 landed
        const float* s = ring + (jy % STG) * SLOTF;
        const long long own = site_of(xc, y);
        float acc = 0.f;
        float4 o0 = *(const float4*)(s + 4 * lane);
        float4 o1 = *(const float4*)(s + 128 + 4 * lane);
        acc = o0.x + o0.y + o0.z + o0.w + o1.x + o1.y + o1.z + o1.w;
        const bool even = ((xc & 1) == 0) && lane < 31;  // x0 = 30k is even: lanes 1,3,..,29
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            if (H) {
                const unsigned w = __float_as_uint(s[256 + 64 * (i - 1) + 2 * lane]) ^ __float_as_uint(acc);
                const unsigned wf = __float_as_uint(s[768 + 32 * (i - 1) + lane]);
                const long long src = site_of(xc - CX(i), y - CY(i));
                const unsigned short fv = ((src & 1) ? (wf >> 16) : (wf & 0xffff)) ^ (unsigned short)i;
                unsigned short* B = (unsigned short*)out.pop;
                if (PAIR) {
                    const unsigned wn = __shfl_down_sync(0xffffffffu, w, 1);
                    const unsigned fn = __shfl_down_sync(0xffffffffu, (unsigned)fv, 1);
                    if (outl && even) {
                        *(uint2*)(B + 2 * (i - 1) * PLANE + 2 * own) = make_uint2(w, wn);
                        *(unsigned*)(B + (15 + i) * PLANE + own) = (unsigned)fv | (fn << 16);
                    }
                } else if (outl) {
                    *(unsigned*)(B + 2 * (i - 1) * PLANE + 2 * own) = w;
                    B[(15 + i) * PLANE + own] = fv;
                }
            } else {
                const float2 p = *(const float2*)(s + 256 + 64 * (i - 1) + 2 * lane);
                const float fv = s[768 + 32 * (i - 1) + lane] * 0.999f;
                const float2 q = make_float2(p.x * 0.999f + acc, p.y);
                float* B = (float*)out.pop;
                if (PAIR) {
                    const float qx = __shfl_down_sync(0xffffffffu, q.x, 1);
                    const float qy = __shfl_down_sync(0xffffffffu, q.y, 1);
                    const float fn = __shfl_down_sync(0xffffffffu, fv, 1);
                    if (outl && even) {
                        *(float4*)(B + 2 * (i - 1) * PLANE + 2 * own) = make_float4(q.x, q.y, qx, qy);
                        *(float2*)(B + (15 + i) * PLANE + own) = make_float2(fv, fn);
                    }
                } else if (outl) {
                    *(float2*)(B + 2 * (i - 1) * PLANE + 2 * own) = q;
                    B[(15 + i) * PLANE + own] = fv;
                }
            }
        }
        if (outl) {
            *(float4*)(out.aux + 4 * own) = make_float4(o0.x * 0.5f, o0.y, o0.z, acc);
            *(float4*)(out.aux + 4 * PLANE + 4 * own) = o1;
            if (H) *(float2*)(out.aux + 8 * PLANE + 2 * own) = *(const float2*)(s + 1024 + 2 * lane);
        }
    }
    cpa_wait<0>();
}

// ---------------------------------------------------------------- V1 / V2
template <typename ST, int STG, bool BULK_OUT, bool PAIR = false>
__global__ void __launch_bounds__(128, 2) v1(Bufs in, Bufs out, const Item* items, int n_items, int* err) {
    using LL = L<ST>;
    constexpr bool H = sizeof(ST) == 2;
    extern __shared__ __align__(128) unsigned char smb[];
    __shared__ __align__(8) uint64_t mbar[4][STG];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int it = blockIdx.x * 4 + warp;
    constexpr int PER_WARP = STG * LL::kSlot + (BULK_OUT ? LL::kOut : 0);
    unsigned char* ring = smb + warp * PER_WARP;
    unsigned char* obuf = ring + STG * LL::kSlot;
    if (lane == 0)
        for (int s = 0; s < STG; ++s) mbar_init(&mbar[warp][s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncwarp();
    if (it >= n_items) return;
    const Item W = items[it];
    const int x0 = W.x0;
    const int R = W.y1 - W.y0 + 2;
    const char* A = (const char*)in.pop;
    // segment k of a slot: (byte offset in slot, global source, bytes)
    auto issue = [&](int j) {
        if (j >= R) return;
        const int y = W.y0 - 1 + j;
        unsigned char* s = ring + (j % STG) * LL::kSlot;
        uint64_t* m = &mbar[warp][j % STG];
        fence_async();
        __syncwarp();
        if (lane == 0) mbar_expect(m, LL::kSlot);
        if (lane < LL::kNseg) {
            int off, bytes;
            const char* src;
            if (lane < 8) {
                const int i = lane + 1;
                const long long st = site_of(x0 - LL::kGH0 - CX(i), y - CY(i));
                // align the start down to the segment granule (the segment
                // covers [x0 - kGH0 - CX, ...) shifted; take the aligned superset)
                const long long a = (st + 0) & (H ? ~3LL : ~1LL);
                src = A + (2 * (long long)(i - 1) * PLANE + 2 * a) * sizeof(ST);
                off = (i - 1) * LL::kGHb;
                bytes = LL::kGHb;
            } else if (lane < 16) {
                const int i = lane - 7;
                const long long st = site_of(x0 - LL::kF0 - CX(i), y - CY(i));
                const long long a = st & (H ? ~7LL : ~3LL);
                src = A + ((15 + i) * PLANE + a) * sizeof(ST);
                off = 8 * LL::kGHb + (i - 1) * LL::kFb;
                bytes = LL::kFb;
            } else if (lane == 16) {
                src = (const char*)(in.aux + 4 * site_of(x0 - 2, y));
                off = 8 * LL::kGHb + 8 * LL::kFb;
                bytes = LL::kOwnb;
            } else if (lane == 17) {
                src = (const char*)(in.aux + 4 * PLANE + 4 * site_of(x0 - 2, y));
                off = 8 * LL::kGHb + 8 * LL::kFb + LL::kOwnb;
                bytes = LL::kOwnb;
            } else {
                src = (const char*)(in.aux + 8 * PLANE + 2 * site_of(x0 - 2, y));
                off = 8 * LL::kGHb + 8 * LL::kFb + 2 * LL::kOwnb;
                bytes = LL::kRefb;
            }
            bulk_g2s(s + off, src, bytes, m);
        }
    };
    // as the step kernel: rows 0..STG-1 in flight, rows 0 and 1 consumed first
#pragma unroll
    for (int j = 0; j < STG; ++j) issue(j);
    float carry = 0.f;
    for (int j = 0; j < 2; ++j) {
        if (!mbar_wait(&mbar[warp][j % STG], (j / STG) & 1)) atomicExch(err, 1);
        carry += *(const float*)(ring + (j % STG) * LL::kSlot + 8 * LL::kGHb + 8 * LL::kFb + 16 * (lane + 2));
    }
    for (int y = W.y0; y < W.y1; ++y) {
        const int jy = y - W.y0 + 1;
        issue(jy + STG - 1);   // into the slot of row jy - 1 (consumed in the previous iteration)
        if (jy + 1 < R) {      // row jy + 1 must land (the step kernel's look-ahead macro row)
            if (!mbar_wait(&mbar[warp][(jy + 1) % STG], ((jy + 1) / STG) & 1)) atomicExch(err, 1);
            carry += *(const float*)(ring + ((jy + 1) % STG) * LL::kSlot + 8 * LL::kGHb + 8 * LL::kFb + 16 * (lane + 2));
        }
        const unsigned char* s = ring + (jy % STG) * LL::kSlot;
        const int xc = x0 + lane;
        const long long own = site_of(xc, y);
        const float4 o0 = *(const float4*)(s + 8 * LL::kGHb + 8 * LL::kFb + 16 * (lane + 2));
        const float4 o1 = *(const float4*)(s + 8 * LL::kGHb + 8 * LL::kFb + LL::kOwnb + 16 * (lane + 2));
        const float acc = o0.x + o0.y + o0.z + o0.w + o1.x + o1.y + o1.z + o1.w + carry;
        if (BULK_OUT) {
            if (y > W.y0) {  // the previous row's bulk stores must have read obuf
                if (lane < LL::kNseg) bulk_wait_read0();
                __syncwarp();
            }
        }
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            // the segment of direction i starts kGH0 (kF0) sites left of x0,
            // aligned down: its start shift relative to x0 - kGH0 - CX(i)
            const long long stg = site_of(x0 - LL::kGH0 - CX(i), y - CY(i));
            const int dg = (int)(stg - (stg & (H ? ~3LL : ~1LL)));
            const long long stf = site_of(x0 - LL::kF0 - CX(i), y - CY(i));
            const int df = (int)(stf - (stf & (H ? ~7LL : ~3LL)));
            const int kg = lane + LL::kGH0 + dg;   // index of this lane's source in the gh segment
            const int kf = lane + LL::kF0 + df;
            if (H) {
                const unsigned w = *(const unsigned*)(s + (i - 1) * LL::kGHb + 4 * kg);
                const unsigned short fv = *(const unsigned short*)(s + 8 * LL::kGHb + (i - 1) * LL::kFb + 2 * kf);
                if (BULK_OUT) {
                    *(unsigned*)(obuf + (i - 1) * 128 + 4 * lane) = w ^ __float_as_uint(acc);
                    *(unsigned short*)(obuf + 1024 + (i - 1) * 64 + 2 * lane) = fv ^ (unsigned short)i;
                } else if (PAIR) {
                    unsigned short* B = (unsigned short*)out.pop;
                    const unsigned a = w ^ __float_as_uint(acc), b = fv ^ (unsigned short)i;
                    const unsigned an = __shfl_down_sync(0xffffffffu, a, 1);
                    const unsigned bn = __shfl_down_sync(0xffffffffu, b, 1);
                    if ((lane & 1) == 0) {
                        *(uint2*)(B + 2 * (i - 1) * PLANE + 2 * own) = make_uint2(a, an);
                        *(unsigned*)(B + (15 + i) * PLANE + own) = b | (bn << 16);
                    }
                } else {
                    unsigned short* B = (unsigned short*)out.pop;
                    *(unsigned*)(B + 2 * (i - 1) * PLANE + 2 * own) = w ^ __float_as_uint(acc);
                    B[(15 + i) * PLANE + own] = fv ^ (unsigned short)i;
                }
            } else {
                const float2 p = *(const float2*)(s + (i - 1) * LL::kGHb + 8 * kg);
                const float fv = *(const float*)(s + 8 * LL::kGHb + (i - 1) * LL::kFb + 4 * kf);
                if (BULK_OUT) {
                    *(float2*)(obuf + (i - 1) * 256 + 8 * lane) = make_float2(p.x * 0.999f + acc, p.y);
                    *(float*)(obuf + 2048 + (i - 1) * 128 + 4 * lane) = fv * 0.999f;
                } else if (PAIR) {
                    float* B = (float*)out.pop;
                    const float qx = p.x * 0.999f + acc, qy = p.y, fq = fv * 0.999f;
                    const float nx_ = __shfl_down_sync(0xffffffffu, qx, 1);
                    const float ny_ = __shfl_down_sync(0xffffffffu, qy, 1);
                    const float nf = __shfl_down_sync(0xffffffffu, fq, 1);
                    if ((lane & 1) == 0) {
                        *(float4*)(B + 2 * (i - 1) * PLANE + 2 * own) = make_float4(qx, qy, nx_, ny_);
                        *(float2*)(B + (15 + i) * PLANE + own) = make_float2(fq, nf);
                    }
                } else {
                    float* B = (float*)out.pop;
                    *(float2*)(B + 2 * (i - 1) * PLANE + 2 * own) = make_float2(p.x * 0.999f + acc, p.y);
                    B[(15 + i) * PLANE + own] = fv * 0.999f;
                }
            }
        }
        const float4 w0 = make_float4(o0.x * 0.5f, o0.y, o0.z, acc);
        if (BULK_OUT) {
            constexpr int ob = H ? 1536 : 3072;
            *(float4*)(obuf + ob + 16 * lane) = w0;
            *(float4*)(obuf + ob + 512 + 16 * lane) = o1;
            if (H) *(float2*)(obuf + ob + 1024 + 8 * lane) =
                *(const float2*)(s + 8 * LL::kGHb + 8 * LL::kFb + 2 * LL::kOwnb + 8 * (lane + 2));
            fence_async();
            __syncwarp();
            if (lane < LL::kNseg) {
                char* dst;
                const unsigned char* src;
                int bytes;
                char* Bp = (char*)out.pop;
                const long long o = site_of(x0, y);
                if (lane < 8) {
                    const int i = lane + 1;
                    dst = Bp + (2 * (long long)(i - 1) * PLANE + 2 * o) * sizeof(ST);
                    src = obuf + (i - 1) * (H ? 128 : 256);
                    bytes = H ? 128 : 256;
                } else if (lane < 16) {
                    const int i = lane - 7;
                    dst = Bp + ((15 + i) * PLANE + o) * sizeof(ST);
                    src = obuf + (H ? 1024 : 2048) + (i - 1) * (H ? 64 : 128);
                    bytes = H ? 64 : 128;
                } else if (lane == 16) {
                    dst = (char*)(out.aux + 4 * o); src = obuf + ob; bytes = 512;
                } else if (lane == 17) {
                    dst = (char*)(out.aux + 4 * PLANE + 4 * o); src = obuf + ob + 512; bytes = 512;
                } else {
                    dst = (char*)(out.aux + 8 * PLANE + 2 * o); src = obuf + ob + 1024; bytes = 256;
                }
                bulk_s2g(dst, src, bytes);
                bulk_commit();
            }
        } else {
            *(float4*)(out.aux + 4 * own) = w0;
            *(float4*)(out.aux + 4 * PLANE + 4 * own) = o1;
            if (H) *(float2*)(out.aux + 8 * PLANE + 2 * own) =
                *(const float2*)(s + 8 * LL::kGHb + 8 * LL::kFb + 2 * LL::kOwnb + 8 * (lane + 2));
        }
    }
    if (BULK_OUT && lane < LL::kNseg) bulk_wait0();
}


// ---------------------------------------------------------------- V3 blocked layout
// Every 32-site block of a row keeps all its planes together:
// pop block (y, xb): [24 planes][32] of ST, aux block: [NA planes][32] floats.
// The ring holds source-row blocks (each loaded once by two bulk copies); the
// pull of row y reads planes of class CY = +1 from block y-1, 0 from y, -1
// from y+1 (no x halo in this copy-only form).
constexpr int NXB = NX / 32;
template <typename ST, int STG>
__global__ void __launch_bounds__(128, 2) v3(Bufs in, Bufs out, const Item* items, int n_items, int* err) {
    constexpr bool H = sizeof(ST) == 2;
    constexpr int NA = H ? 10 : 8;
    constexpr int POPB = 24 * 32 * (int)sizeof(ST), AUXB = NA * 32 * 4, BLK = POPB + AUXB;
    extern __shared__ __align__(128) unsigned char smb[];
    __shared__ __align__(8) uint64_t mbar[4][STG];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int it = blockIdx.x * 4 + warp;
    unsigned char* ring = smb + warp * STG * BLK;
    if (lane == 0)
        for (int q = 0; q < STG; ++q) mbar_init(&mbar[warp][q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncwarp();
    if (it >= n_items) return;
    const Item W = items[it];
    const int xb = W.x0 / 32;
    const int R = W.y1 - W.y0 + 2;  // source rows y0-1 .. y1
    auto blk = [&](int y) { return (long long)(y + 2) * NXB + xb; };
    auto issue = [&](int j) {
        if (j >= R) return;
        const int y = W.y0 - 1 + j;
        unsigned char* sl = ring + (j % STG) * BLK;
        uint64_t* m = &mbar[warp][j % STG];
        fence_async();
        __syncwarp();
        if (lane == 0) {
            mbar_expect(m, BLK);
            bulk_g2s(sl, (const char*)in.pop + blk(y) * POPB, POPB, m);
            bulk_g2s(sl + POPB, (const char*)in.aux + blk(y) * AUXB, AUXB, m);
        }
    };
    for (int j = 0; j < STG; ++j) issue(j);
    for (int j = 0; j < 2; ++j)
        if (!mbar_wait(&mbar[warp][j % STG], (j / STG) & 1)) atomicExch(err, 1);
    for (int y = W.y0; y < W.y1; ++y) {
        const int jy = y - W.y0 + 1;
        if (jy + 1 < R)
            if (!mbar_wait(&mbar[warp][(jy + 1) % STG], ((jy + 1) / STG) & 1)) atomicExch(err, 1);
        const unsigned char* bm = ring + ((jy - 1) % STG) * BLK;
        const unsigned char* b0 = ring + (jy % STG) * BLK;
        const unsigned char* bp = ring + ((jy + 1) % STG) * BLK;
        const float* a0 = (const float*)(b0 + POPB);
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < NA; ++k) acc += a0[k * 32 + lane];
        ST* ob = (ST*)out.pop + blk(y) * (24 * 32);
        float* oa = out.aux + blk(y) * (NA * 32);
#pragma unroll
        for (int q = 0; q < 24; ++q) {
            const int i = q < 16 ? (q >> 1) + 1 : q - 15;  // direction of plane q
            const unsigned char* src = CY(i) > 0 ? bm : (CY(i) < 0 ? bp : b0);
            const int l2 = min(31, max(0, lane - CX(i)));
            const ST v = ((const ST*)src)[q * 32 + l2];
            if constexpr (H) ob[q * 32 + lane] = (ST)(v ^ (ST)q);
            else ob[q * 32 + lane] = v * 0.999f + acc;
        }
#pragma unroll
        for (int k = 0; k < NA; ++k) oa[k * 32 + lane] = a0[k * 32 + lane] * 0.5f;
        __syncwarp();
        issue(jy + STG - 1);  // the slot of row jy - 1, read above
    }
}


// ---------------------------------------------------------------- V4 / V5: blocked layout, pull-row staging
// A ring slot holds what pull row y needs: plane q of the block of source row
// y - CY(dir(q)). V4 copies each plane (24 bulk copies + the own-site block of
// row y); V5 stores the block's planes grouped by CY class (+1, 0, -1), so a
// pull row takes three chunk copies (+ the own-site block). Copy-only: the x
// halo is left out; reads shift inside the padded (V4) or plain (V5) rows.
template <typename ST, int STG, bool CHUNK>
__global__ void __launch_bounds__(128, 2) v45(Bufs in, Bufs out, const Item* items, int n_items, int* err) {
    constexpr bool H = sizeof(ST) == 2;
    constexpr int NA = H ? 10 : 8;
    constexpr int ES = sizeof(ST);
    constexpr int POPB = 24 * 32 * ES, AUXB = NA * 32 * 4;
    constexpr int PAD = 16 / ES;                 // elements before a plane's 32 (16 B)
    constexpr int ROW = CHUNK ? 32 : 32 + 2 * PAD;  // smem elements per plane row
    constexpr int SLOT = 24 * ROW * ES + AUXB;
    extern __shared__ __align__(128) unsigned char smb[];
    __shared__ __align__(8) uint64_t mbar[4][STG];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int it = blockIdx.x * 4 + warp;
    unsigned char* ring = smb + warp * STG * SLOT;
    if (lane == 0)
        for (int q = 0; q < STG; ++q) mbar_init(&mbar[warp][q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncwarp();
    if (it >= n_items) return;
    const Item W = items[it];
    const int xb = W.x0 / 32;
    const int R = W.y1 - W.y0 + 2;  // pull rows y0-1 .. y1
    auto blk = [&](int y) { return (long long)(y + 2) * NXB + xb; };
    // plane q: direction and class. Planes 0..15 are (g,h) rows of direction
    // q/2+1, 16..23 f of direction q-15; CHUNK order: class +1 first.
    auto dir_of = [](int q) { return q < 16 ? (q >> 1) + 1 : q - 15; };
    auto issue = [&](int j) {
        if (j >= R) return;
        const int y = W.y0 - 1 + j;
        unsigned char* sl = ring + (j % STG) * SLOT;
        uint64_t* m = &mbar[warp][j % STG];
        fence_async();
        __syncwarp();
        if (lane == 0) mbar_expect(m, 24 * 32 * ES + AUXB);
        if (CHUNK) {
            // chunk c (c = 0: class +1 from row y-1, 1: class 0 from row y,
            // 2: class -1 from row y+1): 8, 8 and 8 planes (V5 order)
            if (lane < 3) {
                const int yy = y - (1 - lane);
                bulk_g2s(sl + lane * 8 * 32 * ES, (const char*)in.pop + blk(yy) * POPB + lane * 8 * 32 * ES,
                         8 * 32 * ES, m);
            } else if (lane == 3) {
                bulk_g2s(sl + 24 * 32 * ES, (const char*)in.aux + blk(y) * AUXB, AUXB, m);
            }
        } else {
            if (lane < 24) {
                const int yy = y - CY(dir_of(lane));
                bulk_g2s(sl + (lane * ROW + PAD) * ES, (const char*)in.pop + blk(yy) * POPB + lane * 32 * ES,
                         32 * ES, m);
            } else if (lane == 24) {
                bulk_g2s(sl + 24 * ROW * ES, (const char*)in.aux + blk(y) * AUXB, AUXB, m);
            }
        }
    };
    for (int j = 0; j < STG; ++j) issue(j);
    for (int j = 0; j < 2; ++j)
        if (!mbar_wait(&mbar[warp][j % STG], (j / STG) & 1)) atomicExch(err, 1);
    for (int y = W.y0; y < W.y1; ++y) {
        const int jy = y - W.y0 + 1;
        if (jy + 1 < R)
            if (!mbar_wait(&mbar[warp][(jy + 1) % STG], ((jy + 1) / STG) & 1)) atomicExch(err, 1);
        const unsigned char* b0 = ring + (jy % STG) * SLOT;
        const float* a0 = (const float*)(b0 + 24 * ROW * ES);
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < NA; ++k) acc += a0[k * 32 + lane];
        ST* ob = (ST*)out.pop + blk(y) * (24 * 32);
        float* oa = out.aux + blk(y) * (NA * 32);
#pragma unroll
        for (int q = 0; q < 24; ++q) {
            const int i = dir_of(q);
            int k;
            if (CHUNK) k = min(31, max(0, lane - CX(i)));
            else k = lane - CX(i) + PAD;
            const ST v = ((const ST*)b0)[q * ROW + k];
            if constexpr (H) ob[q * 32 + lane] = (ST)(v ^ (ST)q);
            else ob[q * 32 + lane] = v * 0.999f + acc;
        }
#pragma unroll
        for (int k = 0; k < NA; ++k) oa[k * 32 + lane] = a0[k * 32 + lane] * 0.5f;
        __syncwarp();
        issue(jy + STG - 1);
    }
}

// ---------------------------------------------------------------- host
template <typename K>
float time_it(K launch, int reps) {
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a)); CK(cudaEventCreate(&b));
    for (int r = 0; r < 3; ++r) launch(r);
    CK(cudaDeviceSynchronize());
    float best = 1e30f;
    for (int t = 0; t < 3; ++t) {
        CK(cudaEventRecord(a));
        for (int r = 0; r < reps; ++r) launch(r);
        CK(cudaEventRecord(b));
        CK(cudaEventSynchronize(b));
        float ms; CK(cudaEventElapsedTime(&ms, a, b));
        best = std::min(best, ms / reps);
    }
    CK(cudaGetLastError());
    return best * 1e3f;  // us
}

int main(int argc, char** argv) {
    const double peak = argc > 1 ? atof(argv[1]) : 6789.3;
    int sms = 0; CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
    const size_t popb32 = 24 * PLANE * 4, auxb32 = 8 * PLANE * 4;
    const size_t popb16 = 24 * PLANE * 2, auxb16 = 10 * PLANE * 4;
    Bufs b32[2], b16[2];
    for (int k = 0; k < 2; ++k) {
        CK(cudaMalloc(&b32[k].pop, popb32)); CK(cudaMalloc(&b32[k].aux, auxb32));
        CK(cudaMalloc(&b16[k].pop, popb16)); CK(cudaMalloc(&b16[k].aux, auxb16));
        CK(cudaMemset(b32[k].pop, 0, popb32)); CK(cudaMemset(b32[k].aux, 0, auxb32));
        CK(cudaMemset(b16[k].pop, 0, popb16)); CK(cudaMemset(b16[k].aux, 0, auxb16));
    }
    int* err; CK(cudaMalloc(&err, 4)); CK(cudaMemset(err, 0, 4));
    const double sites = (double)NX * NY;
    auto items_for = [&](int w, int rows) {
        std::vector<Item> v;
        for (int y0 = 0; y0 < NY; y0 += rows)
            for (int x0 = 0; x0 < NX; x0 += w) v.push_back({x0, y0, std::min(y0 + rows, NY), 0});
        return v;
    };
    Item* d_items; CK(cudaMalloc(&d_items, sizeof(Item) * 200000));
    auto report = [&](const char* name, float us, double bpl, int n_items, int rows) {
        printf("%-28s rows=%3d items=%6d  %7.2f us  %8.1f GB/s  %.3f of peak\n", name, rows, n_items, us,
               bpl * sites / (us * 1e-6) / 1e9, bpl * sites / (us * 1e-6) / 1e9 / peak);
    };
    std::vector<int> rows_list = {8, 16, 32};
    const char* only = argc > 2 ? argv[2] : "";
    if (argc > 3) rows_list = {atoi(argv[3])};
    const int reps = argc > 4 ? atoi(argv[4]) : 20;
    auto want = [&](const char* n) { return !*only || strstr(n, only) != nullptr; };
    for (int rows : rows_list) {
        auto it30 = items_for(30, rows);
        auto it32 = items_for(32, rows);
        auto run_v0 = [&](auto kern, int stg, bool h, const char* name) {
            if (!want(name)) return;
            CK(cudaMemcpy(d_items, it30.data(), sizeof(Item) * it30.size(), cudaMemcpyHostToDevice));
            const int n = (int)it30.size(), blocks = (n + 3) / 4;
            const int smem = 4 * stg * (h ? 34 : 32) * 32 * 4;
            CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            Bufs* b = h ? b16 : b32;
            float t = time_it([&](int r) { kern<<<blocks, 128, smem>>>(b[r & 1], b[(r & 1) ^ 1], d_items, n); }, reps);
            report(name, t, h ? 176 : 256, n, rows);
        };
        auto run_v1 = [&](auto kern, int stg, bool h, const char* name) {
            if (!want(name)) return;
            CK(cudaMemcpy(d_items, it32.data(), sizeof(Item) * it32.size(), cudaMemcpyHostToDevice));
            const int n = (int)it32.size(), blocks = (n + 3) / 4;
            const int smem = 4 * stg * (h ? L<unsigned short>::kSlot : L<float>::kSlot);
            CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            Bufs* b = h ? b16 : b32;
            float t = time_it([&](int r) { kern<<<blocks, 128, smem>>>(b[r & 1], b[(r & 1) ^ 1], d_items, n, err); }, reps);
            report(name, t, h ? 176 : 256, n, rows);
        };
        run_v0(v0<float, 3, false>, 3, false, "v0f32_s3");
        run_v0(v0<float, 4, false>, 4, false, "v0f32_s4");
        run_v0(v0<float, 5, false>, 5, false, "v0f32_s5");
        run_v0(v0<unsigned short, 3, false>, 3, true, "v0f16_s3");
        run_v0(v0<unsigned short, 4, false>, 4, true, "v0f16_s4");
        run_v0(v0<unsigned short, 5, false>, 5, true, "v0f16_s5");
        run_v0(v0<unsigned short, 6, false>, 6, true, "v0f16_s6");
        run_v1(v1<float, 3, false>, 3, false, "v1f32_s3");
        run_v1(v1<float, 4, false>, 4, false, "v1f32_s4");
        run_v1(v1<float, 5, false>, 5, false, "v1f32_s5");
        run_v1(v1<unsigned short, 3, false>, 3, true, "v1f16_s3");
        run_v1(v1<unsigned short, 4, false>, 4, true, "v1f16_s4");
        run_v1(v1<unsigned short, 6, false>, 6, true, "v1f16_s6");
        run_v1(v1<unsigned short, 8, false>, 8, true, "v1f16_s8");
        auto run_v3 = [&](auto kern, int stg, bool h, const char* name) {
            if (!want(name)) return;
            CK(cudaMemcpy(d_items, it32.data(), sizeof(Item) * it32.size(), cudaMemcpyHostToDevice));
            const int n = (int)it32.size(), blocks = (n + 3) / 4;
            const int blk = h ? 24 * 32 * 2 + 10 * 32 * 4 : 24 * 32 * 4 + 8 * 32 * 4;
            const int smem = 4 * stg * blk;
            CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            Bufs* b = h ? b16 : b32;
            float t = time_it([&](int r) { kern<<<blocks, 128, smem>>>(b[r & 1], b[(r & 1) ^ 1], d_items, n, err); }, reps);
            report(name, t, h ? 176 : 256, n, rows);
        };
        run_v3(v3<float, 4>, 4, false, "v3f32_s4");
        run_v3(v3<float, 6>, 6, false, "v3f32_s6");
        run_v3(v3<unsigned short, 4>, 4, true, "v3f16_s4");
        run_v3(v3<unsigned short, 6>, 6, true, "v3f16_s6");
        run_v3(v3<unsigned short, 8>, 8, true, "v3f16_s8");
        auto run_v45 = [&](auto kern, int stg, bool h, bool chunk, const char* name) {
            if (!want(name)) return;
            CK(cudaMemcpy(d_items, it32.data(), sizeof(Item) * it32.size(), cudaMemcpyHostToDevice));
            const int n = (int)it32.size(), blocks = (n + 3) / 4;
            const int es = h ? 2 : 4, pad = 16 / es, row = chunk ? 32 : 32 + 2 * pad;
            const int slot = 24 * row * es + (h ? 10 : 8) * 32 * 4;
            const int smem = 4 * stg * slot;
            CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            Bufs* b = h ? b16 : b32;
            float t = time_it([&](int r) { kern<<<blocks, 128, smem>>>(b[r & 1], b[(r & 1) ^ 1], d_items, n, err); }, reps);
            report(name, t, h ? 176 : 256, n, rows);
        };
        run_v45(v45<float, 3, false>, 3, false, false, "v4f32_s3");
        run_v45(v45<float, 4, false>, 4, false, false, "v4f32_s4");
        run_v45(v45<unsigned short, 3, false>, 3, true, false, "v4f16_s3");
        run_v45(v45<unsigned short, 4, false>, 4, true, false, "v4f16_s4");
        run_v45(v45<unsigned short, 6, false>, 6, true, false, "v4f16_s6");
        run_v45(v45<float, 3, true>, 3, false, true, "v5f32_s3");
        run_v45(v45<float, 4, true>, 4, false, true, "v5f32_s4");
        run_v45(v45<unsigned short, 3, true>, 3, true, true, "v5f16_s3");
        run_v45(v45<unsigned short, 4, true>, 4, true, true, "v5f16_s4");
        run_v45(v45<unsigned short, 6, true>, 6, true, true, "v5f16_s6");
    }
    int herr = 0; CK(cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost));
    printf("sms=%d err=%d\n", sms, herr);
    return herr;
}
