// me9_tile.cuh -- the T = 9 warp-strip tile of the dense template-matching motion estimation
// (Sec. 2.2): for every pixel of a tile and one past frame the vector v in [-R, R]^2 (p + v inside
// the frame) of least masked SAD, ties in the order |v|_1, v_y, v_x.  Shared by the ME launches
// (me.cu) and the fused ME + checks launch (cc.cu); each translation unit gets its own copy.
#pragma once
#include <type_traits>

#include "rfsr_internal.h"

namespace rfsr {
namespace {
namespace me9k {

constexpr int NVMAX = (2 * kMaxRadius + 1) * (2 * kMaxRadius + 1);

// Candidates of [-R, R]^2 sorted by (|v|_1, v_y, v_x): enumerate |v|_1 = L, then v_y ascending,
// then v_x ascending (-|v_x| before +|v_x|).
__device__ __forceinline__ void build_tie_order(short2 *vord, int R)
{
    if (threadIdx.x != 0) return;
    int n = 0;
    for (int L = 0; L <= 2 * R; ++L)
        for (int vy = -R; vy <= R; ++vy) {
            const int ax = L - (vy < 0 ? -vy : vy);
            if (ax < 0 || ax > R) continue;
            vord[n++] = make_short2((short)vy, (short)-ax);
            if (ax != 0) vord[n++] = make_short2((short)vy, (short)ax);
        }
}

// ---------------------------------------------------------------------------------------------
// T = 9: warp-strip kernel with byte SIMD.  Lane l of a warp owns four adjacent columns (one
// 32-bit word of bytes) of a 128-column strip, the warp owns 8 output rows, the CTA 4 warps (8 in
// one of the batched tile shapes).
// For each candidate the lane walks the 16 rows of D_v its outputs need: one aligned load of the
// past-frame word from the byte-shifted copy of its column phase, __vabsdiffu4, AND with the
// mask, and running vertical sums kept as two packed 16-bit words (columns 0,2 and 1,3).  The
// 9-column horizontal sums take the left and right lanes' vertical sums (four shuffles) and a few
// packed adds.  The running argmin is packed too: two outputs per word, a guard-bit compare
// (cost + 0x7fff - new has its lane MSB set iff new < cost), a sign-replicating prmt into a lane
// mask and two bit selects.  Candidates run in tie order with strict improvement, so the first
// minimum in tie order wins.  Lanes 0 and 31 only feed their neighbours: a strip yields 120
// output columns.  CTAs whose candidates all stay inside the frame run a loop without the
// border masks.
// ---------------------------------------------------------------------------------------------
// The template tile of a CTA is WARPS strips of 8 rows x 120 columns; its search window (the
// staged past-frame rows) is the tile plus the template half and the radius on each side.
constexpr int S_ROWS = 8;                  // output rows per warp
constexpr int S_OUTW = 120;                // output columns per CTA
constexpr int S_DROWS = S_ROWS + 8;        // D rows per warp (T = 9)
constexpr int S_RWORDS = (128 + 2 * kMaxRadius + 3) / 4 + 1;   // words per staged row
template <int WARPS> __host__ __device__ constexpr int s_nt() { return 32 * WARPS; }
template <int WARPS, int ROWS = S_ROWS> __host__ __device__ constexpr int s_outh() { return ROWS * WARPS; }   // tile rows
template <int WARPS, int ROWS = S_ROWS> __host__ __device__ constexpr int s_rrows() { return ROWS * WARPS + 8 + 2 * kMaxRadius; }

// lane masks from the guard bits of a packed pair: 0xffff in each 16-bit lane whose bit 15 (lo)
// or bit 31 (hi) is set (prmt's default mode replicates the sign bit when a selector's msb is set)
__device__ __forceinline__ uint32_t lane_mask(uint32_t t)
{
    uint32_t m;
    asm("prmt.b32 %0, %1, 0, 0xbb99;" : "=r"(m) : "r"(t));
    return m;
}

// a * b + c on the integer multiply-add unit.  With b = 1 (or -1, both held in registers whose
// value the compiler cannot see) it is an addition (subtraction) that runs on the FMA pipe, which
// the byte-SIMD work of these kernels leaves idle, instead of taking another ALU slot.
__device__ __forceinline__ uint32_t imad(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// The staged past-frame window in four byte-shifted copies: copy j, word w of a row holds row
// bytes 4 w + j .. 4 w + j + 3, so the word a lane compares at any column is one aligned load.
template <int WARPS, int ROWS = S_ROWS>
struct Smem9 {
    uint32_t rf[4][s_rrows<WARPS, ROWS>() * S_RWORDS];
    short2 vord[NVMAX];
};

template <int WARPS, int ROWS = S_ROWS>
__device__ __forceinline__ void me9_tile(Smem9<WARPS, ROWS> &sm, const FrameTask &t, int tbx, int tby, int k)
{
    constexpr int S_NT = s_nt<WARPS>(), S_OUTH = s_outh<WARPS, ROWS>();
    constexpr int DROWS = ROWS + 8;                       // D rows per warp (T = 9)
    const int x0 = tbx * S_OUTW, y0 = tby * S_OUTH;
    const int H = t.H, W = t.W, R = t.R;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (*t.status) return;
    const uint8_t *__restrict__ ref = t.ref_rec[k];

    // past frame around the CTA: rows y0-4-R .., columns x0-4-R .., clamped coordinates.  A word
    // inside the frame is one aligned 32-bit load when the plane's rows and the window start are
    // 4-byte aligned (W % 4 == 0, R % 4 == 0); words across a border take clamped bytes.
    const int rx0 = x0 - 4 - R, ry0 = y0 - 4 - R;
    const int nrows = S_OUTH + 8 + 2 * R;
    const bool al_ref = ((W | rx0) & 3) == 0 && ((uintptr_t)ref & 3) == 0;
    for (int i = threadIdx.x; i < nrows * S_RWORDS; i += S_NT) {
        const int r = i / S_RWORDS, w = i - r * S_RWORDS;
        const uint8_t *row = ref + (size_t)min(max(ry0 + r, 0), H - 1) * W;
        const int gx = rx0 + 4 * w;
        uint32_t v = 0;
        if (al_ref && gx >= 0 && gx + 4 <= W) {
            v = *reinterpret_cast<const uint32_t *>(row + gx);
        } else {
#pragma unroll
            for (int b = 0; b < 4; ++b) v |= (uint32_t)row[min(max(gx + b, 0), W - 1)] << (8 * b);
        }
        sm.rf[0][i] = v;
    }
    build_tie_order(sm.vord, R);

    // current frame: this lane's 16 rows of 4 columns (masked samples, byte masks; 0 outside),
    // one aligned 32-bit load per plane and row where the word lies inside a 4-byte aligned frame
    const int cx = x0 - 4 + 4 * lane;                     // first column of the lane's word
    const int cy0 = y0 + ROWS * warp - 4;               // first D row of the warp
    const bool al_cur = (W & 3) == 0 && (((uintptr_t)t.cur_smp | (uintptr_t)t.cur_msk) & 3) == 0 &&
                        cx >= 0 && cx + 4 <= W;           // cx is a multiple of 4
    uint32_t cs[DROWS], cmk[DROWS];
#pragma unroll
    for (int i = 0; i < DROWS; ++i) {
        const int y = cy0 + i;
        uint32_t a = 0, m = 0;
        if (y >= 0 && y < H) {
            const size_t ro = (size_t)y * W;
            if (al_cur) {
                a = *reinterpret_cast<const uint32_t *>(t.cur_smp + ro + cx);
                m = *reinterpret_cast<const uint32_t *>(t.cur_msk + ro + cx);
            } else {
#pragma unroll
                for (int b = 0; b < 4; b += 2) {
                    const int x = cx + b;
                    if (x >= 0 && x < W) {    // W even, x even: pixel pairs never straddle
                        a |= (uint32_t)(*reinterpret_cast<const uint16_t *>(t.cur_smp + ro + x)) << (8 * b);
                        m |= (uint32_t)(*reinterpret_cast<const uint16_t *>(t.cur_msk + ro + x)) << (8 * b);
                    }
                }
            }
        }
        cs[i] = a;
        cmk[i] = m;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * nrows * (S_RWORDS - 1); i += S_NT) {
        const int j = 1 + i / (nrows * (S_RWORDS - 1));
        const int rem = i - (j - 1) * nrows * (S_RWORDS - 1);
        const int r = rem / (S_RWORDS - 1), w = rem - r * (S_RWORDS - 1);
        sm.rf[j][r * S_RWORDS + w] =
            __funnelshift_r(sm.rf[0][r * S_RWORDS + w], sm.rf[0][r * S_RWORDS + w + 1], 8 * j);
    }
    __syncthreads();

    // border handling: candidates with p + v outside the frame are not allowed
    const bool border = (x0 - 4 - R < 0) || (x0 + 124 + R > W) || (y0 - R < 0) || (y0 + S_OUTH + R > H);
    uint32_t best02[ROWS], best13[ROWS], idx02[ROWS], idx13[ROWS];
#pragma unroll
    for (int j = 0; j < ROWS; ++j) {
        best02[j] = best13[j] = 0x7fff7fffu;
        idx02[j] = idx13[j] = 0u;
    }
    const int nv = (2 * R + 1) * (2 * R + 1);
    const int oy = y0 + ROWS * warp;                     // first output row of the warp
    const uint32_t one = (uint32_t)(W > 0), m1 = 0u - one;  // 1 and -1 (W > 0 always)
    // the candidate loop, instantiated for border CTAs (some p + v outside the frame) and for
    // interior ones (no invalid-column or invalid-row masking at all)
    auto candidates = [&](auto border_tag) {
        constexpr bool BORDER = decltype(border_tag)::value;
        for (int o = 0; o < nv; ++o) {
            const short2 v = sm.vord[o];
            const int vy = v.x, vx = v.y;
            const int sh = (vx + R) & 3, q = (vx + R) >> 2;
            const uint32_t *rrow = sm.rf[sh] + (ROWS * warp + vy + R) * S_RWORDS + lane + q;
            uint32_t inv02 = 0, inv13 = 0;                     // lanes of invalid columns -> 0x7fff
            if constexpr (BORDER) {
                const int c0 = cx + vx;
                inv02 = ((unsigned)(c0) >= (unsigned)W ? 0x7fffu : 0u) |
                        ((unsigned)(c0 + 2) >= (unsigned)W ? 0x7fff0000u : 0u);
                inv13 = ((unsigned)(c0 + 1) >= (unsigned)W ? 0x7fffu : 0u) |
                        ((unsigned)(c0 + 3) >= (unsigned)W ? 0x7fff0000u : 0u);
            }
            uint32_t lo = 0, hi = 0;                           // vertical sums, columns (0,2) (1,3)
            uint32_t dlo[DROWS], dhi[DROWS];
            const uint32_t o2 = (uint32_t)o * 0x00010001u;
    #pragma unroll
            for (int i = 0; i < DROWS; ++i) {
                const uint32_t d4 = __vabsdiffu4(cs[i], rrow[i * S_RWORDS]) & cmk[i];
                dlo[i] = __byte_perm(d4, 0u, 0x4240);
                dhi[i] = __byte_perm(d4, 0u, 0x4341);
                lo = imad(dlo[i], one, lo);
                hi = imad(dhi[i], one, hi);
                if (i >= 9) {
                    lo = imad(dlo[i - 9], m1, lo);
                    hi = imad(dhi[i - 9], m1, hi);
                }
                if (i >= 8) {
                    const int j = i - 8;                       // output row of this window
                    const uint32_t Q = imad(hi, one, lo);      // (c0+c1, c2+c3)
                    const uint32_t Ql = __shfl_up_sync(0xffffffffu, Q, 1);
                    const uint32_t lol = __shfl_up_sync(0xffffffffu, lo, 1);
                    const uint32_t Qr = __shfl_down_sync(0xffffffffu, Q, 1);
                    const uint32_t lor = __shfl_down_sync(0xffffffffu, lo, 1);
                    const uint32_t A = __byte_perm(Ql, Q, 0x5432);   // (left c-2+c-1, c0+c1)
                    const uint32_t B = __byte_perm(Q, Qr, 0x5432);   // (c2+c3, right c4+c5)
                    uint32_t h02 = imad(lor, one, imad(imad(B, one, Q), one, imad(A, one, Ql)));  // (H0, H2)
                    uint32_t h13 = imad(imad(lol, m1, Qr), one, imad(lor, m1, h02));         // (H1, H3)
                    if constexpr (BORDER) {
                        const uint32_t rinv = (unsigned)(oy + j + vy) >= (unsigned)H ? 0x7fff7fffu : 0u;
                        h02 |= inv02 | rinv;
                        h13 |= inv13 | rinv;
                    }
                    const uint32_t m02 = lane_mask(best02[j] + 0x7fff7fffu - h02);
                    const uint32_t m13 = lane_mask(best13[j] + 0x7fff7fffu - h13);
                    best02[j] = (best02[j] & ~m02) | (h02 & m02);
                    idx02[j] = (idx02[j] & ~m02) | (o2 & m02);
                    best13[j] = (best13[j] & ~m13) | (h13 & m13);
                    idx13[j] = (idx13[j] & ~m13) | (o2 & m13);
                }
            }
        }
    };
    if (border) candidates(std::true_type{});
    else candidates(std::false_type{});
    if (lane == 0 || lane == 31) return;
    char2 *mv = reinterpret_cast<char2 *>(t.mv[k]);
#pragma unroll
    for (int j = 0; j < ROWS; ++j) {
        const int y = oy + j;
        if (y >= H) continue;
        const uint32_t id[4] = {idx02[j] & 0xffffu, idx13[j] & 0xffffu, idx02[j] >> 16, idx13[j] >> 16};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int x = cx + c;
            if (x < W) {
                const short2 v = sm.vord[id[c]];
                mv[(size_t)y * W + x] = make_char2((signed char)v.x, (signed char)v.y);
            }
        }
    }
}

}  // namespace me9k
}  // namespace
}  // namespace rfsr
