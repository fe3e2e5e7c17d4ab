// lbm_block.cuh -- the block step kernel: one warp advances one 32-site
// column of row blocks (the blocked layout's unit, see lbm_internal.h) over a
// segment of rows. Included by lbm_kernels.cu inside its anonymous namespace,
// after the per-site pieces it reuses (pulls, local_macro, the stencils,
// site_update_to); not a standalone header.
//
// Per row ("pull row" y) the warp needs, for every direction i, the
// populations that arrive at its 32 sites: those of row y - c_iy. In the
// blocked layout they are three contiguous chunks (P of row y - 1, Z of row y,
// M of row y + 1) plus the own-site block of row y, so four bulk copies
// (cp.async.bulk, one lane each, completing on one mbarrier) stage a row;
// next to a wall the chunk of the row behind it is replaced by the opposite
// chunk of row y itself (bounce-back, same order). The columns on either
// side of the block (x0 - 2, x0 - 1, x0 + w, x0 + w + 1; periodic x) come as
// small per-lane cp.async pieces arriving on the same mbarrier. The local
// macroscopic fields of the two side columns, which the stencils of the edge
// lanes need, are computed by two lanes in a second pass and kept in a small
// per-warp ring in shared memory. Every offset inside the staged row is a
// compile-time constant plus the lane.

// ---- mbarrier, bulk copies ---------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* m, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* m, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(m)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* m, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_addr(m)), "r"(parity)
        : "memory");
    return ok != 0;
}
// The arrival of this thread on *m once all its earlier cp.async copies have
// landed (the barrier's count includes it: .noinc).
__device__ __forceinline__ void mbar_arrive_cp_async(uint64_t* m) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(m)) : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* m) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(m))
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Polls of a staged row before a warp gives up (each poll waits a bounded
// time in hardware; far beyond any copy's latency).
constexpr int kMbarPolls = 1 << 22;

// ---- one staged row in shared memory (bytes) -------------------------------
template <typename ST>
struct BlockSlot {
    static constexpr int E = (int)sizeof(ST);
    static constexpr int kPop = 16;  // chunks P, Z, M (a lane's read one site left stays inside)
    static constexpr int kOwn = kPop + kPopBlock * E;   // (g_0, h_0', f_0, f_l), (phi u, p, S), [refs]
    static constexpr int kOwnBytes = E == 4 ? 1024 : 1280;
    static constexpr int kHaloGH = kOwn + kOwnBytes + 16;  // [side][dir 1..8][near, far] pairs
    static constexpr int kHaloF = kHaloGH + 2 * 8 * 2 * 2 * E;  // 6 words: dirs 1,5,8 left, 3,6,7 right
    static constexpr int kHaloO0 = kHaloF + 32;                 // [side] float4
    static constexpr int kHaloO1 = kHaloO0 + 32;
    static constexpr int kHaloR = kHaloO1 + 32;                 // [side] float2
    static constexpr int kBytes = kHaloR + 16;
    static constexpr unsigned kTx = kPopBlock * E + kOwnBytes;  // bytes of the four bulk copies
    static constexpr int kPieces = E == 4 ? 32 : 34;            // side-column copies per row
    static_assert(kBytes % 16 == 0 && kOwn % 16 == 0 && kHaloO0 % 16 == 0, "slot alignment");
};
// Side-column macroscopic ring: [ring row][side][field] with fields phi, rho,
// T, p, S and phi one column further out (rows next to a wall only).
constexpr int kHaloFields = 6;
constexpr int kBlockStg = 3;  // staged rows per warp

// Per-warp dynamic shared memory of the block kernel (bytes): ring slots,
// mbarriers, the side-column ring and one float per lane for the item's mdot.
template <typename ST>
struct BlockWarp {
    static constexpr int kMbar = kBlockStg * BlockSlot<ST>::kBytes;
    static constexpr int kHring = kMbar + 8 * kBlockStg;
    static constexpr int kMd = kHring + 4 * 3 * 2 * kHaloFields;
    static constexpr int kBytes = (kMd + 4 * 32 + 15) / 16 * 16;
};

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// The three chunk positions of a staged row: which row and chunk each holds.
struct RowSrc {
    int rr;          // the pull row (wrapped)
    int rowP, chP;   // position P: chunk P of row rr-1, or chunk M of rr at a wall below
    int rowM, chM;   // position M: chunk M of row rr+1, or chunk P of rr at a wall above
    bool bP, bM;     // bounced positions
};
__device__ __forceinline__ RowSrc row_src(int y, int ny, bool py) {
    RowSrc r;
    r.rr = wrapi(y, ny);
    r.bP = !py && r.rr == 0;
    r.bM = !py && r.rr == ny - 1;
    r.rowP = r.bP ? r.rr : wrapi(r.rr - 1, ny);
    r.chP = r.bP ? kChunkM : kChunkP;
    r.rowM = r.bM ? r.rr : wrapi(r.rr + 1, ny);
    r.chM = r.bM ? kChunkP : kChunkM;
    return r;
}

// Direction i's link bounces at a wall in this row; then it is read at the
// lane's own column, else one column over (c_ix).
__device__ __forceinline__ bool dir_bounced(int i, const RowSrc& r) {
    const int pos = chunk_of(i);
    return (pos == kChunkP && r.bP) || (pos == kChunkM && r.bM);
}
__device__ __forceinline__ int dir_shift(int i, const RowSrc& r) { return dir_bounced(i, r) ? 0 : CX(i); }

// Wetting ghost (Eqs. 39-41) behind a wall from the adjacent row a and the
// next one b, given each one's neighbours on both sides.
__device__ __forceinline__ float wet_ghost(float a, float am, float ap, float bm, float bp,
                                           float tan_w) {
    const float d0 = 0.5f * (ap - am);
    const float d1 = 0.5f * (bp - bm);
    return a + tan_w * fabsf(1.5f * d0 - 0.5f * d1);
}

// Populations of a staged row as site_update reads them: g and h of
// direction i from the chunk (decoded for 16-bit storage with the site's
// references), f from registers; the edge lanes take the side columns; h of
// a bounced link at a Dirichlet wall becomes anti-bounce-back.
template <typename ST>
struct BlockPops {
    const unsigned char* sl;
    int lane, w;
    RowSrc r;
    int dmask;     // bit i: h_i arrives through a Dirichlet wall
    float abb;     // Cp_ref T_w
    Ref ref;       // 16-bit storage: the site's references
    float Cpref;
    const float* f;
    __device__ __forceinline__ float2 pair(int i) const {
        using BS = BlockSlot<ST>;
        const int sh = dir_shift(i, r);
        const int k = lane - sh;
        const unsigned char* p = sl + BS::kPop + (gh_off(i) + 2 * k) * BS::E;
        if (sh > 0 && lane == 0) p = sl + BS::kHaloGH + ((0 * 8 + (i - 1)) * 2 + 0) * 2 * BS::E;
        if (sh < 0 && lane == w - 1) p = sl + BS::kHaloGH + ((1 * 8 + (i - 1)) * 2 + 0) * 2 * BS::E;
        if constexpr (sizeof(ST) == 4) {
            return *reinterpret_cast<const float2*>(p);
        } else {
            const unsigned wd = *reinterpret_cast<const unsigned*>(p);
            return make_float2(Bits16<ST>::add_lo(wd, WGT(i) * ref.phi),
                               Bits16<ST>::add_hi(wd, WGT(i) * Cpref * ref.T));
        }
    }
    __device__ __forceinline__ float4 own0() const {
        return *reinterpret_cast<const float4*>(sl + BlockSlot<ST>::kOwn + 16 * lane);
    }
    __device__ __forceinline__ float G(int i) const { return i == 0 ? own0().x : pair(i).x; }
    __device__ __forceinline__ float H(int i) const {
        if (i == 0) return own0().y;
        const float v = pair(i).y;
        return ((dmask >> i) & 1) ? -v + 2.0f * WGT(i) * abb : v;
    }
    __device__ __forceinline__ float F(int i) const { return f[i]; }
};

// f of a staged row at the lane's site (the edge lanes from the side
// columns), decoded for 16-bit storage with the source pressures pref
// (pref[0]: the site's own, for bounced links).
template <typename ST>
__device__ __forceinline__ void block_f(const unsigned char* sl, int lane, int w, const RowSrc& r,
                                        int parL, int parR, const float* pref, float f[9]) {
    using BS = BlockSlot<ST>;
    f[0] = *reinterpret_cast<const float*>(sl + BS::kOwn + 16 * lane + 8);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const int sh = dir_shift(i, r);
        const int k = lane - sh;
        const int fo = BS::kPop + (f_off(i) + k) * BS::E;
        // side words: dirs 1, 5, 8 on the left (0..2), 3, 6, 7 on the right (3..5)
        constexpr int jl[9] = {0, 0, 0, 0, 0, 1, 0, 0, 2}, jr[9] = {0, 0, 0, 3, 0, 0, 4, 5, 0};
        if constexpr (sizeof(ST) == 4) {
            const float* p = reinterpret_cast<const float*>(sl + fo);
            if (sh > 0 && lane == 0) p = reinterpret_cast<const float*>(sl + BS::kHaloF + 4 * jl[i]);
            if (sh < 0 && lane == w - 1) p = reinterpret_cast<const float*>(sl + BS::kHaloF + 4 * jr[i]);
            f[i] = *p;
        } else {
            unsigned short raw = *reinterpret_cast<const unsigned short*>(sl + fo);
            if (sh > 0 && lane == 0) {
                const unsigned wd = *reinterpret_cast<const unsigned*>(sl + BS::kHaloF + 4 * jl[i]);
                raw = (unsigned short)(parL ? (wd >> 16) : (wd & 0xffffu));
            }
            if (sh < 0 && lane == w - 1) {
                const unsigned wd = *reinterpret_cast<const unsigned*>(sl + BS::kHaloF + 4 * jr[i]);
                raw = (unsigned short)(parR ? (wd >> 16) : (wd & 0xffffu));
            }
            // a bounced link carries the site's own population: its own pressure
            f[i] = Bits16<ST>::fma_lo_2m12((unsigned)raw, f_rest(i, dir_bounced(i, r) ? pref[0] : pref[i]));
        }
    }
}

// The local macroscopic step at one site from the g and h a staged row
// delivers there, read through `at(i)` -> pointer of the (g_i, h_i) pair.
template <typename ST, typename At>
__device__ __forceinline__ Macro block_macro(const Phys& P, At at, const float4& o0, const Ref& ref,
                                             int dmask, float abb) {
    float g[9], h[9];
    g[0] = o0.x;
    h[0] = o0.y;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const unsigned char* p = at(i);
        if constexpr (sizeof(ST) == 4) {
            const float2 v = *reinterpret_cast<const float2*>(p);
            g[i] = v.x;
            h[i] = v.y;
        } else {
            const unsigned wd = *reinterpret_cast<const unsigned*>(p);
            g[i] = Bits16<ST>::add_lo(wd, WGT(i) * ref.phi);
            h[i] = Bits16<ST>::add_hi(wd, WGT(i) * P.Cpref * ref.T);
        }
        if ((dmask >> i) & 1) h[i] = -h[i] + 2.0f * WGT(i) * abb;
    }
    return local_macro(P, g, h, o0.w);
}

// One warp advances block item W (columns [x0, x0 + w), rows [y0, y1)) by one
// step. ring: kBlockStg slots; mbar: kBlockStg barriers (initialised, count
// 33, phases tracked in *phase); hring: the side-column ring; mdsm: 32 floats.
// Returns false when a staged row never completed (the error word is raised).
template <bool OBS, typename ST, bool NC>
__device__ __forceinline__ bool block_item(const Inst* __restrict__ insts, const Item& W, int parity,
                                           double* __restrict__ partials, unsigned char* ring,
                                           uint64_t* mbar, unsigned& phase, float* hring,
                                           float* mdsm, int* err) {
    using BS = BlockSlot<ST>;
    constexpr bool kHalf = sizeof(ST) != 4;
    const int lane = threadIdx.x & 31;
    const Inst& I = insts[W.inst];
    const Phys P = load_phys(I);
    const int nx = I.nx, ny = I.ny, flags = I.flags;
    const bool py = (flags & kPeriodicY) != 0;
    const int nxb = I.pitch >> 5;
    const int x0 = W.x0, xb = x0 >> 5;
    const int w = min(32, nx - x0);
    const bool out_lane = lane < w;
    const ST* A = static_cast<const ST*>(I.pop[parity]);
    const float* Aaux = I.aux[parity];
    const float abb = P.Cpref * P.Tw;
    // side columns (periodic x)
    const int cL1 = wrapi(x0 - 1, nx), cL2 = wrapi(x0 - 2, nx);
    const int cR1 = wrapi(x0 + w, nx), cR2 = wrapi(x0 + w + 1, nx);
    const int parL = cL1 & 1, parR = cR1 & 1;  // 16-bit f words: which half
    const int y0 = W.y0, R = W.y1 - y0 + 2;    // staged rows y0 - 1 .. y1
    const bool has_lo = y0 >= 1 || py, has_hi = W.y1 < ny || py;

    auto slot = [&](int j) { return ring + (j % kBlockStg) * BS::kBytes; };
    auto staged = [&](int j) { return j < R && (j > 0 || has_lo) && (j < R - 1 || has_hi); };

    // ---- staging of ring index j (pull row y0 - 1 + j) ----
    auto issue = [&](int j) {
        if (!staged(j)) return;
        const RowSrc r = row_src(y0 - 1 + j, ny, py);
        unsigned char* sl = slot(j);
        uint64_t* m = mbar + (j % kBlockStg);
        fence_proxy_async_smem();  // the slot's previous reads (generic) before the copies (async)
        __syncwarp();
        if (lane == 0) mbar_expect_tx(m, BS::kTx);
        const long long bP = ((long long)r.rowP * nxb + xb) * kPopBlock;
        const long long bZ = ((long long)r.rr * nxb + xb) * kPopBlock;
        const long long bM = ((long long)r.rowM * nxb + xb) * kPopBlock;
        if (lane == 0) bulk_load(sl + BS::kPop + kChunkP * BS::E, A + bP + r.chP, 288 * BS::E, m);
        if (lane == 1) bulk_load(sl + BS::kPop + kChunkZ * BS::E, A + bZ + kChunkZ, 192 * BS::E, m);
        if (lane == 2) bulk_load(sl + BS::kPop + kChunkM * BS::E, A + bM + r.chM, 288 * BS::E, m);
        if (lane == 3)
            bulk_load(sl + BS::kOwn, Aaux + ((long long)r.rr * nxb + xb) * kAuxBlock, BS::kOwnBytes, m);
        // side-column pieces: piece q of this lane (and q + 32 for 16-bit storage)
        auto piece = [&](int q) {
            // q 0..15: (g, h) of direction (q & 7) + 1 at the near column of side q >> 3;
            // 16..21: the far column for dirs 1, 5, 8 (left) and 3, 6, 7 (right);
            // 22..27: f at the near column, same directions; 28..31: own0, own1
            // left / right; 32, 33: references left / right
            int side, d = 0, kind, col;
            // the directions whose far column is needed: 1, 5, 8 (left), 3, 6, 7
            // (right), chosen without an array indexed at run time
            auto far_dir = [](int t) {
                return t == 0 ? 1 : (t == 1 ? 5 : (t == 2 ? 8 : (t == 3 ? 3 : (t == 4 ? 6 : 7))));
            };
            if (q < 16) { side = q >> 3; d = (q & 7) + 1; kind = 0; col = 0; }
            else if (q < 22) { side = q >= 19; d = far_dir(q - 16); kind = 0; col = 1; }
            else if (q < 28) { side = q >= 25; d = far_dir(q - 22); kind = 1; col = 0; }
            else if (q < 32) { side = q & 1; kind = q < 30 ? 2 : 3; col = 0; }
            else { side = q & 1; kind = 4; col = 0; }
            const int c = side == 0 ? (col ? cL2 : cL1) : (col ? cR2 : cR1);
            const int cb = c >> 5, cl = c & 31;
            if (kind <= 1) {
                const int pos = chunk_of(d);
                const int row = pos == kChunkP ? r.rowP : (pos == kChunkM ? r.rowM : r.rr);
                const int ch = pos == kChunkP ? r.chP : (pos == kChunkM ? r.chM : kChunkZ);
                const long long blk = ((long long)row * nxb + cb) * kPopBlock;
                if (kind == 0) {
                    const long long e = blk + ch + 64 * chunk_k(d) + 2 * cl;
                    unsigned char* dst = sl + BS::kHaloGH + ((side * 8 + (d - 1)) * 2 + col) * 2 * BS::E;
                    if constexpr (kHalf) cp_async4(reinterpret_cast<float*>(dst), reinterpret_cast<const float*>(A + e));
                    else cp_async8(reinterpret_cast<float*>(dst), reinterpret_cast<const float*>(A + e));
                } else {
                    long long e = blk + ch + 64 * chunk_n(d) + 32 * chunk_k(d) + cl;
                    if constexpr (kHalf) e &= ~1LL;  // the aligned word holding it
                    unsigned char* dst = sl + BS::kHaloF + 4 * (q - 22);
                    cp_async4(reinterpret_cast<float*>(dst), reinterpret_cast<const float*>(A + e));
                }
            } else {
                const long long a = ((long long)r.rr * nxb + cb) * kAuxBlock;
                if (kind == 2) cp_async16(reinterpret_cast<float*>(sl + BS::kHaloO0 + 16 * side), Aaux + a + 4 * cl);
                else if (kind == 3) cp_async16(reinterpret_cast<float*>(sl + BS::kHaloO1 + 16 * side), Aaux + a + 128 + 4 * cl);
                else cp_async8(reinterpret_cast<float*>(sl + BS::kHaloR + 8 * side), Aaux + a + 256 + 2 * cl);
            }
        };
        piece(lane);
        if (kHalf && lane < BS::kPieces - 32) piece(32 + lane);
        mbar_arrive_cp_async(m);
    };
    // wait for ring index j; false (error raised) after kMbarPolls polls
    auto land = [&](int j) {
        if (!staged(j)) return true;
        const int s = j % kBlockStg;
        const unsigned par = (phase >> s) & 1u;
        for (int k = 0; k < kMbarPolls; ++k) {
            if (mbar_try_wait(mbar + s, par)) {
                phase ^= 1u << s;
                return true;
            }
        }
        atomicExch(err, 2);
        return false;
    };
    // on giving up: wait (bounded) for every row still in flight, then return
    auto drain = [&](int from, int to) {
        for (int j = from; j < to; ++j) land(j);
    };

    // ---- macroscopic fields of a staged row ----
    // the lane's site (rows behind a wall are never asked for)
    auto own_macro = [&](int j, Macro& m, float& p, float& S, Ref& ref) {
        const unsigned char* sl = slot(j);
        const RowSrc r = row_src(y0 - 1 + j, ny, py);
        const float4 o0 = *reinterpret_cast<const float4*>(sl + BS::kOwn + 16 * lane);
        const float4 o1 = *reinterpret_cast<const float4*>(sl + BS::kOwn + 512 + 16 * lane);
        ref = Ref{0.f, 0.f};
        if constexpr (kHalf) {
            const float2 rf = *reinterpret_cast<const float2*>(sl + BS::kOwn + 1024 + 8 * lane);
            ref = Ref{rf.x, rf.y};
        }
        const int dmask = (r.bP && (flags & kDirYlo) ? (1 << 2) | (1 << 5) | (1 << 6) : 0) |
                          (r.bM && (flags & kDirYhi) ? (1 << 4) | (1 << 7) | (1 << 8) : 0);
        m = block_macro<ST>(P, [&](int i) {
            const int sh = dir_shift(i, r);
            const unsigned char* q = sl + BS::kPop + (gh_off(i) + 2 * (lane - sh)) * BS::E;
            if (sh > 0 && lane == 0) q = sl + BS::kHaloGH + ((0 * 8 + (i - 1)) * 2 + 0) * 2 * BS::E;
            if (sh < 0 && lane == w - 1) q = sl + BS::kHaloGH + ((1 * 8 + (i - 1)) * 2 + 0) * 2 * BS::E;
            return q;
        }, o0, ref, dmask, abb);
        p = o1.z;
        S = o1.w;
    };
    // the two side columns (lane 0: x0 - 1, lane 1: x0 + w) into hring
    auto side_macro = [&](int j) {
        if (lane < 2) {
            const int side = lane;
            const unsigned char* sl = slot(j);
            const RowSrc r = row_src(y0 - 1 + j, ny, py);
            const float4 o0 = *reinterpret_cast<const float4*>(sl + BS::kHaloO0 + 16 * side);
            const float4 o1 = *reinterpret_cast<const float4*>(sl + BS::kHaloO1 + 16 * side);
            Ref ref{0.f, 0.f};
            if constexpr (kHalf) {
                const float2 rf = *reinterpret_cast<const float2*>(sl + BS::kHaloR + 8 * side);
                ref = Ref{rf.x, rf.y};
            }
            const int dmask = (r.bP && (flags & kDirYlo) ? (1 << 2) | (1 << 5) | (1 << 6) : 0) |
                              (r.bM && (flags & kDirYhi) ? (1 << 4) | (1 << 7) | (1 << 8) : 0);
            const Macro m = block_macro<ST>(P, [&](int i) {
                const int sh = dir_shift(i, r);
                // the source column of the side site: one further out (far),
                // the side column itself (near), or the block's edge site
                const unsigned char* q;
                if (sh == 0) q = sl + BS::kHaloGH + ((side * 8 + (i - 1)) * 2 + 0) * 2 * BS::E;
                else if ((sh > 0) == (side == 0)) q = sl + BS::kHaloGH + ((side * 8 + (i - 1)) * 2 + 1) * 2 * BS::E;
                else q = sl + BS::kPop + (gh_off(i) + 2 * (side == 0 ? 0 : w - 1)) * BS::E;
                return q;
            }, o0, ref, dmask, abb);
            float* h = hring + ((j % 3) * 2 + side) * kHaloFields;
            h[0] = m.phi;
            h[1] = m.rho;
            h[2] = m.T;
            h[3] = o1.z;
            h[4] = o1.w;
            // phi one column further out, for the wetting ghost of the side
            // column (rows next to a wall only): from global memory
            const int rr = r.rr;
            if (!py && (rr <= 1 || rr >= ny - 2)) {
                LatT<NC> l;
                l.A = reinterpret_cast<const float*>(A);
                l.Aaux = Aaux;
                l.plane = (int)I.plane; l.nx = nx; l.ny = ny; l.pitch = I.pitch; l.flags = flags;
                const int xo = side == 0 ? cL2 : cR2;
                const int idx = rr * I.pitch + xo;
                Ref rf{0.f, 0.f};
                if constexpr (kHalf) { rf.phi = ldAux(l, 5, idx); rf.T = ldAux(l, 6, idx); }
                float gg[9], hh[9];
                pull_set<0, ST>(l, xo, rr, abb, gg, rf, P.Cpref);
                pull_set<1, ST>(l, xo, rr, abb, hh, rf, P.Cpref);
                h[5] = local_macro(P, gg, hh, ldAux(l, 0, idx)).phi;
            }
        }
    };
    // side-column value of field k at ring index j (0 left, 1 right)
    auto hv = [&](int j, int side, int k) { return hring[((j % 3) * 2 + side) * kHaloFields + k]; };

    RowObs ob;
    if (OBS) ob.zero();
    float col_fs = 0.f;
    mdsm[lane] = 0.f;

    // ---- prologue: rows y0 - 1 and y0 ----
#pragma unroll 1
    for (int j = 0; j < kBlockStg; ++j) issue(j);
    if (!land(0) || !land(1)) { drain(2, kBlockStg); return false; }
    float phm = 0.f, ph0, php = 0.f, rhm = 0.f, rh0, rhp = 0.f;
    float pm = 0.f, p0, pp = 0.f, Sm = 0.f, S0, Sp = 0.f;
    float tm = 0.f, t0, tp = 0.f;
    Macro mO;
    Ref rO;
    own_macro(1, mO, p0, S0, rO);
    side_macro(1);
    ph0 = mO.phi; rh0 = mO.rho; t0 = mO.T;
    if (has_lo) {
        Macro mm;
        Ref rr_;
        own_macro(0, mm, pm, Sm, rr_);
        side_macro(0);
        phm = mm.phi; rhm = mm.rho; tm = mm.T;
    }
    __syncwarp();

    for (int y = y0; y < W.y1; ++y) {
        const int jy = y - y0 + 1;
        __syncwarp();  // every lane is done with the previous row (slot, side ring)
        issue(jy + kBlockStg - 1);  // into the slot of row y - 1, read in the previous iteration
        if (!land(jy + 1)) { drain(jy + 2, jy + kBlockStg); return false; }
        const unsigned char* sl = slot(jy);
        const RowSrc r0 = row_src(y, ny, py);
        const float4 o1 = *reinterpret_cast<const float4*>(sl + BS::kOwn + 512 + 16 * lane);
        const float phiux_p = o1.x, phiuy_p = o1.y;

        // row y + 1: the lanes' sites and the side columns
        Macro mN;
        Ref rN{0.f, 0.f};
        const bool top_wall = !(y + 1 < ny || py);
        const bool bottom_wall = y == 0 && !py;
        if (!top_wall) {
            own_macro(jy + 1, mN, pp, Sp, rN);
            side_macro(jy + 1);
            php = mN.phi; rhp = mN.rho; tp = mN.T;
        }
        __syncwarp();
        // neighbour of value v at row ring index j: the lane beside, or the
        // side column for the block's edge lanes (field k of hring)
        auto left = [&](float v, float side_v) {
            const float s = __shfl_up_sync(0xffffffffu, v, 1);
            return lane == 0 ? side_v : s;
        };
        auto right = [&](float v, float side_v) {
            const float s = __shfl_down_sync(0xffffffffu, v, 1);
            return lane == w - 1 ? side_v : s;
        };
        // side-column windows (rows y - 1, y, y + 1) of phi, rho, p, S, T;
        // ghost rows behind a wall: wetting for phi, copies for the rest
        float sPhi[2][3], sRho[2][3], sP[2][3], sS[2][3], sT[2][3];
#pragma unroll
        for (int sd = 0; sd < 2; ++sd) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int j = jy - 1 + q;
                const bool ghost = (q == 0 && bottom_wall) || (q == 2 && top_wall);
                const int jj = ghost ? jy : j;
                sPhi[sd][q] = hv(jj, sd, 0);
                sRho[sd][q] = hv(jj, sd, 1);
                sT[sd][q] = hv(jj, sd, 2);
                sP[sd][q] = hv(jj, sd, 3);
                sS[sd][q] = hv(jj, sd, 4);
            }
        }
        if (top_wall) {
            // row ny lies behind the top wall: ghost from rows ny-1 and ny-2
            php = wet_ghost(ph0, left(ph0, sPhi[0][1]), right(ph0, sPhi[1][1]),
                            left(phm, sPhi[0][0]), right(phm, sPhi[1][0]), P.tan_w);
            rhp = rh0; pp = p0; Sp = S0; tp = t0;
#pragma unroll
            for (int sd = 0; sd < 2; ++sd) {
                // the side column's ghost: its neighbours are the edge site
                // and phi one column further out
                const float in1 = __shfl_sync(0xffffffffu, ph0, sd == 0 ? 0 : w - 1);
                const float in2 = __shfl_sync(0xffffffffu, phm, sd == 0 ? 0 : w - 1);
                const float out1 = hv(jy, sd, 5), out2 = hv(jy - 1, sd, 5);
                // left side column: out is its left neighbour, in its right one
                sPhi[sd][2] = sd == 0 ? wet_ghost(sPhi[sd][1], out1, in1, out2, in2, P.tan_w)
                                      : wet_ghost(sPhi[sd][1], in1, out1, in2, out2, P.tan_w);
            }
        }
        if (bottom_wall) {
            phm = wet_ghost(ph0, left(ph0, sPhi[0][1]), right(ph0, sPhi[1][1]),
                            left(php, sPhi[0][2]), right(php, sPhi[1][2]), P.tan_w);
            rhm = rh0; pm = p0; Sm = S0; tm = t0;
#pragma unroll
            for (int sd = 0; sd < 2; ++sd) {
                const float in1 = __shfl_sync(0xffffffffu, ph0, sd == 0 ? 0 : w - 1);
                const float in2 = __shfl_sync(0xffffffffu, php, sd == 0 ? 0 : w - 1);
                const float out1 = hv(jy, sd, 5), out2 = hv(jy + 1, sd, 5);
                sPhi[sd][0] = sd == 0 ? wet_ghost(sPhi[sd][1], out1, in1, out2, in2, P.tan_w)
                                      : wet_ghost(sPhi[sd][1], in1, out1, in2, out2, P.tan_w);
            }
        }

        // Eq. 38 from column sums; the edge lanes' outer columns from the
        // side windows
        Stencil st;
        {
            auto cs = [&](float m_, float c_, float p_) { return col_sums(m_, c_, p_); };
            auto sides = [&](const ColSums& v, const float sv[2][3], ColSums& L, ColSums& Rr) {
                const ColSums sl_ = cs(sv[0][0], sv[0][1], sv[0][2]);
                const ColSums sr_ = cs(sv[1][0], sv[1][1], sv[1][2]);
                L.A = left(v.A, sl_.A);
                L.D = left(v.D, sl_.D);
                Rr.A = right(v.A, sr_.A);
                Rr.D = right(v.D, sr_.D);
            };
            ColSums L, Rr;
            const ColSums cph = cs(phm, ph0, php);
            sides(cph, sPhi, L, Rr);
            grad_cols(L, cph, Rr, st.gphx, st.gphy);
            const float sph = php + phm;
            st.lph = lap_cols(left(ph0, sPhi[0][1]), ph0, right(ph0, sPhi[1][1]),
                              left(sph, sPhi[0][2] + sPhi[0][0]), sph,
                              right(sph, sPhi[1][2] + sPhi[1][0]));
            const ColSums crh = cs(rhm, rh0, rhp);
            sides(crh, sRho, L, Rr);
            grad_cols(L, crh, Rr, st.grx, st.gry);
            const ColSums cpp = cs(pm, p0, pp);
            sides(cpp, sP, L, Rr);
            grad_cols(L, cpp, Rr, st.gpx, st.gpy);
            const ColSums cSS = cs(Sm, S0, Sp);
            sides(cSS, sS, L, Rr);
            grad_cols(L, cSS, Rr, st.gSx, st.gSy);
        }

        // 16-bit storage: the source pressures of the pulled f and the
        // references of the sites each outgoing population streams into
        float pref[9];
        Ref dref[9];
        if constexpr (kHalf) {
            pref[0] = p0;
            dref[0] = Ref{ph0, t0};
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                const int cy = CY(i), cx = CX(i);
                const int qs = cy > 0 ? 0 : (cy < 0 ? 2 : 1);  // source row y - cy
                const float ps = cy > 0 ? pm : (cy < 0 ? pp : p0);
                pref[i] = cx > 0 ? left(ps, sP[0][qs]) : (cx < 0 ? right(ps, sP[1][qs]) : ps);
                const int qd = cy > 0 ? 2 : (cy < 0 ? 0 : 1);  // destination row y + cy
                const float vp = cy > 0 ? php : (cy < 0 ? phm : ph0);
                const float vt = cy > 0 ? tp : (cy < 0 ? tm : t0);
                const float dp = cx > 0 ? right(vp, sPhi[1][qd]) : (cx < 0 ? left(vp, sPhi[0][qd]) : vp);
                const float dt = cx > 0 ? right(vt, sT[1][qd]) : (cx < 0 ? left(vt, sT[0][qd]) : vt);
                const bool wall = (cy > 0 && top_wall) || (cy < 0 && bottom_wall);
                dref[i] = wall ? Ref{ph0, t0} : Ref{dp, dt};
            }
        }
        float f[9];
        block_f<ST>(sl, lane, w, r0, parL, parR, pref, f);

        if (out_lane) {
            const int dmask = (r0.bP && (flags & kDirYlo) ? (1 << 2) | (1 << 5) | (1 << 6) : 0) |
                              (r0.bM && (flags & kDirYhi) ? (1 << 4) | (1 << 7) | (1 << 8) : 0);
            const long long ob_blk = (long long)(y * nxb + xb);
            BlockStore out{static_cast<ST*>(I.pop[parity ^ 1]) + ob_blk * kPopBlock,
                           I.aux[parity ^ 1] + ob_blk * kAuxBlock, lane};
            site_update_to<OBS, ST>(P, flags, mO,
                                    BlockPops<ST>{sl, lane, w, r0, dmask, abb, rO, P.Cpref, f},
                                    phiux_p, phiuy_p, st, out, x0 + lane == nx / 2, y == ny / 2,
                                    ob, dref);
            mdsm[lane] += mO.mdot;
            if (OBS) col_fs += mO.fs;
        }
        if (OBS) ob.flush(lane);

        // advance the window
        phm = ph0; ph0 = php; rhm = rh0; rh0 = rhp;
        pm = p0; p0 = pp; Sm = S0; S0 = Sp;
        tm = t0; t0 = tp;
        mO = mN;
        rO = rN;
    }

    if (OBS && RowObs::carried(lane) >= 0)
        partials[(long long)RowObs::carried(lane) * I.part_stride + W.part] = ob.total();
    double* const macc = insts[W.inst].macc;
    if (macc) {
        float v = mdsm[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) macc[W.part] += (double)v;
    }
    if (OBS && I.prof && out_lane) atomicAdd(I.prof + x0 + lane, (double)col_fs);
    return true;
}
