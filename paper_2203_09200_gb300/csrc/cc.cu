// cc.cu -- consistency checks and projection (Sec. 2.2, Sec. 3.1).
//
// For each pixel p of frame t and each past frame t-k (k = 1..K):
//   v~  = component-wise 3x3 median of the ME field (Eq. (1), border replicated) when the mode
//         includes NNC, else the raw vector;  q = p + v~
//   MEASURED        if p is measured in frame t
//   NOT_PROJECTABLE if q is outside the frame or not measured in frame t-k (only measurements
//                   are projected, Sec. 2.2)
//   NNC_REJECT      if the NNC is on and some in-frame 4-neighbour u has |v~(p)-v~(u)|_1 > 1
//                   (Sec. 3.1.2)
//   CHECK_REJECT    if the reverse check fails:
//                     FRMC: some reverse vector -v~+d, d in {-7,-3,-1,0,1,3,7}^2, has a strictly
//                           lower cost than d = 0 (Sec. 3.1.1, Fig. 2c)
//                     RMC:  the same with d in [-Rc, Rc]^2 (Fig. 2b)
//                     RME:  the reverse motion vector found at q is not -v~ (Sec. 2.2)
//                   the reverse cost of d is C(p+d, v~-d): the current-frame template slides
//                   around p while the past-frame patch around q stays fixed; costs are compared
//                   as exact mean absolute differences SAD/n (cross multiplication)
//   ACCEPT          otherwise: psum(p) += f_sub_{t-k}(q), pcnt(p) += 1
// The projected value psum/pcnt is the average over the past frames that project (Sec. 2.2).
// NNC runs first and the reverse check only for NNC survivors (the combination of Sec. 3.1.2).
//
// GB300 design: one CTA per 32x32 pixel tile, all past frames in one launch.  The current frame
// around the tile (template + check halo) is staged once in shared memory as (masked samples,
// byte mask) word pairs in four byte-shifted copies, so that a template row at any column is
// three aligned 8-byte loads; the template counts n are computed once per tile.  Per past frame the
// CTA stages the ME field with a 2-pixel halo and the past frame around the tile (for interior
// tiles fetched with cp.async during the previous past frame's checks), computes the median field
// once, decides every pixel, and compacts the pixels that need a reverse check into a list.  For
// FRMC (T = 9) the vector most listed pixels share is checked by box sums over the tile
// (box_checks9).  For the other listed pixels a warp takes one pixel at a time: the past-frame
// patch around q sits in registers, lane 0 scores d = 0 and the other lanes split the remaining
// offsets, each costing T rows of (AND, byte SAD); a warp vote ends the check as soon as a
// candidate beats d = 0.  The current frame's copies use a row stride of 19 and a copy stride of
// 12 mod 16 units, and the offsets are dealt to lanes (per column phase, nearest first) so that
// the 16 lanes of each half-warp read 16 distinct bank pairs for every template word.
#include <algorithm>
#include <atomic>
#include <type_traits>

#include "me9_tile.cuh"
#include "rfsr_internal.h"

namespace rfsr {

namespace {

constexpr int TP = 32;                        // tile side (pixels)
constexpr int NT = 256;                       // threads per CTA
constexpr int NW = NT / 32;                   // warps per CTA
constexpr int HC = 16;                        // staged halo: |d| <= 9 plus template half <= 5,
                                              // rounded up so the region starts word aligned
constexpr int RS = TP + 2 * HC;               // staged region side (64)
constexpr int NWD = RS / 4 + 1;               // data words per staged row (+1 feeds the shifted copies)
constexpr int RWD = NWD;                      // past frame: row stride (words)
constexpr int CPY = RS * RWD + 8;             // past frame: words per shifted copy
// Current frame (the templates the reverse checks slide): (masked samples, byte mask) word pairs,
// one 8-byte unit per region word, row stride 19 and copy stride 12 (mod 16) units.  A warp's
// 8-byte loads are served per half-warp; with the lane order below the 16 lanes of a half-warp,
// each scoring one offset d of the same pixel, read 16 distinct bank pairs for every template
// word.
constexpr int RWDC = 19;
constexpr int CPYC = RS * RWDC + 12;
constexpr int NS = TP + 2 * kMaxRadius;       // source-count plane side (tile +- 9)
constexpr int MT = TP + 4;                    // ME field tile with a 2-pixel halo
constexpr int MD = TP + 2;                    // median field with a 1-pixel halo
constexpr int PPT = TP * TP / NT;             // pixels owned per thread
constexpr int MSEG = 5;                       // medians per thread task (one row, consecutive)
constexpr int MNSEG = (MD + MSEG - 1) / MSEG; // tasks per median row
static_assert(MD * MNSEG <= NT, "the median field is one pass of the CTA");
// Box-sum FRMC checks (T = 9)
constexpr int BOX_MIN = 64;                   // listed pixels of one vector that pay for a box pass
                                              // (1080p checks: 0.553 ms at 64 and 96, 0.559 at 128,
                                              // 0.623 at 192)
constexpr int HS = 2 * kMaxRadius + 1;        // side of the vector histogram
constexpr int NLMAX = TP * TP * 3 / 4;        // listed pixels of a tile at most (the unmeasured)

// FRMC offsets {-7,-3,-1,0,1,3,7}[i] (Sec. 3.1.1): 0 at i = 3, +-(2^|i-3| - 1) elsewhere
__host__ __device__ constexpr int frmc_offset(int i)
{
    return i == 3 ? 0 : (i < 3 ? -((1 << (3 - i)) - 1) : (1 << (i - 3)) - 1);
}

// Lane order of the reverse-check candidates.  Candidates are indexed row-major in their window
// (FRMC: 7 iy + ix over the offsets above; RMC: side iy + ix, d = (iy - Rc, ix - Rc)).  For each
// column phase (px + HC - h) & 3 of the checked pixel they are dealt into rounds of 32 lanes so
// that no two candidates of a round start their template word in the same bank of the
// current-frame layout: taken in increasing |d|_1 (row-major within a distance), the i-th
// candidate of bank b goes to round i.  A round then reads every template word in one
// shared-memory wavefront; the centre d = 0 is lane 0 of round 0, and the nearest offsets -- the
// likeliest to beat it when the vector is wrong -- fill round 0, so rejections end early.
constexpr int MAXROUND = 16;                  // RMC with Rc = 9 needs 12
constexpr uint16_t NOCAND = 0xffff;
constexpr int NORDER = 1 + kMaxRadius;        // FRMC, then RMC with Rc = 1..9

struct alignas(16) CandOrder {            // copied to shared memory in 16-byte words
    uint16_t lane[4][MAXROUND][32];
    uint32_t nround[4];
};
static_assert(sizeof(CandOrder) % 16 == 0, "CandOrder is copied in 16-byte words");

__host__ __device__ constexpr int cand_dy(int c, bool frmc, int Rc)
{
    return frmc ? frmc_offset(c / 7) : c / (2 * Rc + 1) - Rc;
}

__host__ __device__ constexpr int cand_dx(int c, bool frmc, int Rc)
{
    return frmc ? frmc_offset(c % 7) : c % (2 * Rc + 1) - Rc;
}

// bank pair (8-byte unit mod 16) of a candidate's first template word
constexpr int cand_bank(int c, int ph, bool frmc, int Rc)
{
    const int v = ph + cand_dx(c, frmc, Rc), dy = cand_dy(c, frmc, Rc);
    return ((((v & 3) * CPYC + dy * RWDC + (v >> 2)) % 16) + 16) % 16;
}

// Half-round i of bank pair b holds the i-th candidate (in increasing |d|_1) that starts there;
// round r is half-rounds 2r (lanes 0..15) and 2r + 1 (lanes 16..31).
constexpr void build_order(CandOrder &o, bool frmc, int Rc)
{
    const int side = frmc ? 7 : 2 * Rc + 1, n = side * side, lmax = frmc ? 14 : 2 * Rc;
    for (int ph = 0; ph < 4; ++ph) {
        uint8_t taken[16] = {}, fill[2 * MAXROUND] = {};
        for (int r = 0; r < MAXROUND; ++r)
            for (int l = 0; l < 32; ++l) o.lane[ph][r][l] = NOCAND;
        uint32_t nr = 0;
        for (int L = 0; L <= lmax; ++L)
            for (int c = 0; c < n; ++c) {
                const int dy = cand_dy(c, frmc, Rc), dx = cand_dx(c, frmc, Rc);
                if ((dy < 0 ? -dy : dy) + (dx < 0 ? -dx : dx) != L) continue;
                const int hr = taken[cand_bank(c, ph, frmc, Rc)]++;
                if (hr >= 2 * MAXROUND) {                      // does not fit: order_ok fails
                    o.nround[ph] = MAXROUND + 1;
                    return;
                }
                o.lane[ph][hr / 2][16 * (hr & 1) + fill[hr]++] = (uint16_t)c;
                nr = (uint32_t)hr / 2 + 1 > nr ? (uint32_t)hr / 2 + 1 : nr;
            }
        o.nround[ph] = nr;
    }
}

// every candidate placed once, the centre first, distinct bank pairs in every half-warp
constexpr bool order_ok(const CandOrder &o, bool frmc, int Rc)
{
    const int side = frmc ? 7 : 2 * Rc + 1, n = side * side;
    for (int ph = 0; ph < 4; ++ph) {
        if (o.nround[ph] > MAXROUND || o.lane[ph][0][0] != n / 2) return false;
        int placed = 0;
        for (int r = 0; r < MAXROUND; ++r)
            for (int half = 0; half < 2; ++half) {
                bool seen[16] = {};
                for (int l = 16 * half; l < 16 * half + 16; ++l) {
                    const int c = o.lane[ph][r][l];
                    if (c == NOCAND) continue;
                    ++placed;
                    if (seen[cand_bank(c, ph, frmc, Rc)]) return false;
                    seen[cand_bank(c, ph, frmc, Rc)] = true;
                }
            }
        if (placed != n) return false;
    }
    return true;
}

constexpr bool frmc_order_ok()
{
    CandOrder o{};
    build_order(o, true, 0);
    return order_ok(o, true, 0) && o.nround[0] == 2 && o.nround[1] == 2 && o.nround[2] == 2 &&
           o.nround[3] == 2;
}
static_assert(frmc_order_ok(), "FRMC lane order: two rounds without shared bank pairs");

__device__ CandOrder g_order[NORDER];      // written once per device by init_cc

struct Smem {
    uint2 csm[4 * CPYC];          // (masked samples, byte mask) words, byte-shifted copies
    uint32_t rf[4 * CPY];         // past frame (clamped coordinates), byte-shifted copies
    uint8_t nsrc[NS][NS];         // measured pixels in the template around each source
    uint32_t mv[MT][MT];          // ME field, (v_y + 16, v_x + 16) as 16-bit halves
    uint32_t md[MD][MD];          // its 3x3 median, the same packing
    uint16_t list[TP * TP];       // tile pixels that need a reverse check
    uint8_t rej[TP * TP];
    CandOrder ord;                // reverse-check lane order of this tile's mode
    uint32_t e0n0[TP][TP];        // box checks: cost | count << 16 of d = 0 per tile pixel
    uint16_t ecand[NW][TP][TP];   // box checks: each warp's current candidate cost per tile pixel
    uint16_t blist[TP * TP];      // box checks: listed pixels whose vector is the box vector
    uint32_t be0n0[NLMAX];        // box checks: e0n0 of entry e (read without bank conflicts)
    uint16_t bnoff[NLMAX];        // box checks: offset of entry e's own source in nsrc
    uint32_t rejb[32];            // box checks: rejected bits of blist entries e (word e % 32)
    uint32_t mvraw[MT * MT / 2];  // the next past frame's ME field around the tile (raw char2
                                  // pairs), fetched asynchronously during the current one's checks
    uint32_t rfraw[RS * NWD];     // the next past frame around the tile (raw words), likewise
    int hist[HS * HS];            // listed pixels per filtered vector; once the box vector is
                                  // chosen, the listed pixels with other vectors (plist)
    int boxv;                     // vector (histogram bin) checked by box sums, -1: none
    int nlist;
    int nblist;
    int nplist;
};
static_assert(offsetof(Smem, e0n0) % 16 == 0, "d = 0 costs are read in 16-byte words");
static_assert(offsetof(Smem, ecand) % 8 == 0, "candidate costs are written in 8-byte words");

static_assert(offsetof(Smem, ord) % 16 == 0, "the lane order is written in 16-byte words");

__device__ __forceinline__ int iabs(int v) { return v < 0 ? -v : v; }

// the listed pixels left to the per-pixel checks after a box pass (the histogram is dead by then;
// at most NLMAX - BOX_MIN entries)
__device__ __forceinline__ uint16_t *plist(Smem &sm) { return reinterpret_cast<uint16_t *>(sm.hist); }
static_assert((NLMAX - BOX_MIN) * sizeof(uint16_t) <= sizeof(Smem::hist), "plist fits the histogram");

// Motion vectors in shared memory are (v_y + 128, v_x + 128) as the low and high 16-bit halves
// of a word, so that the median and the neighbour test run on both components at once
// (min.u16x2 / max.u16x2 are single instructions).  The offset keeps both halves positive, so
// subtracting packed words never borrows across the halves; the median commutes with it.  The
// ME field stores a vector as two signed bytes (v_y, v_x); XOR 0x80 turns each into v + 128 and a
// byte permute spreads the pair into the halves.
constexpr int MV_BIAS = 128;
// the vector whose bytes sit at bytes 2j, 2j + 1 of w (j = 0, 1)
__device__ __forceinline__ uint32_t pack_mv(uint32_t w, int j)
{
    return __byte_perm(w ^ 0x80808080u, 0u, 0x4140u + 0x0202u * (unsigned)j);
}
__device__ __forceinline__ int mv_y(uint32_t w) { return (int)(w & 0xffffu) - MV_BIAS; }
__device__ __forceinline__ int mv_x(uint32_t w) { return (int)(w >> 16) - MV_BIAS; }
__device__ __forceinline__ uint32_t pmin(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t pmax(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ void pswap(uint32_t &a, uint32_t &b)
{
    const uint32_t lo = pmin(a, b), hi = pmax(a, b);
    a = lo;
    b = hi;
}
__device__ __forceinline__ uint32_t pmed3(uint32_t a, uint32_t b, uint32_t c)
{
    return pmax(pmin(a, b), pmin(pmax(a, b), c));
}
// Component-wise median of the nine packed vectors of three sorted triples (lo <= mid <= hi per
// half): the median of (largest minimum, median of medians, smallest maximum).  This holds for
// any split of the nine into triples, ties included, so the triples may be the columns of the
// 3x3 window, each sorted once and shared by the three windows that contain it.
struct Sorted3 {
    uint32_t lo, mid, hi;
};
__device__ __forceinline__ Sorted3 psort3(uint32_t a, uint32_t b, uint32_t c)
{
    pswap(a, b);
    pswap(b, c);
    pswap(a, b);
    return {a, b, c};
}
__device__ __forceinline__ uint32_t pmedian9(const Sorted3 &a, const Sorted3 &b, const Sorted3 &c)
{
    const uint32_t lo = __vimax3_u16x2(a.lo, b.lo, c.lo);
    const uint32_t hi = __vimin3_u16x2(a.hi, b.hi, c.hi);
    return pmed3(lo, pmed3(a.mid, b.mid, c.mid), hi);
}
// |a_y - b_y| + |a_x - b_x| <= 1 for packed vectors: max - min per half is |a - b| (no borrow
// between the halves: each half of the maximum is at least that of the minimum, as unsigned
// numbers); times 0x10001 puts the sum of the halves in the high half
__device__ __forceinline__ bool near1(uint32_t a, uint32_t b)
{
    const uint32_t d = pmax(a, b) - pmin(a, b);
    return d * 0x10001u < 0x20000u;
}

// Stage the past frame around the tile (rows y0-HC.., cols x0-HC.., clamped coordinates) as copy
// 0 of four byte-shifted copies (copy j, word w of a row holds region bytes 4w+j .. 4w+j+3; the
// others follow from it in shift_past).  A word inside the frame is one aligned 32-bit load when
// the rows are 4-byte aligned (the region starts at a multiple of 4); words across a border take
// clamped bytes.
__device__ void stage_past0(uint32_t *dst, const uint8_t *__restrict__ src, int H, int W, int y0, int x0)
{
    const bool al = (W & 3) == 0 && ((uintptr_t)src & 3) == 0;
    for (int i = threadIdx.x; i < RS * NWD; i += NT) {
        const int r = i / NWD, w = i - r * NWD;
        const int gy = y0 - HC + r, gx = x0 - HC + 4 * w;
        uint32_t v = 0;
        const uint8_t *row = src + (size_t)min(max(gy, 0), H - 1) * W;
        if (al && gx >= 0 && gx + 4 <= W) {
            v = *reinterpret_cast<const uint32_t *>(row + gx);
        } else {
#pragma unroll
            for (int b = 0; b < 4; ++b) v |= (uint32_t)row[min(max(gx + b, 0), W - 1)] << (8 * b);
        }
        dst[r * RWD + w] = v;
    }
}

// the byte-shifted copies 1..3 from copy 0 (after a barrier that follows stage_past0)
__device__ void shift_past(uint32_t *dst)
{
    for (int i = threadIdx.x; i < 3 * RS * (NWD - 1); i += NT) {
        const int j = 1 + i / (RS * (NWD - 1));
        const int rem = i - (j - 1) * RS * (NWD - 1);
        const int r = rem / (NWD - 1), w = rem - r * (NWD - 1);
        dst[j * CPY + r * RWD + w] = __funnelshift_r(dst[r * RWD + w], dst[r * RWD + w + 1], 8 * j);
    }
}

// Stage the current frame around the tile as (masked samples, byte mask) word pairs in four
// byte-shifted copies (copy j, unit w of a row holds region bytes 4w+j .. 4w+j+3 of both planes;
// 0 outside the frame).
__device__ void stage_current(uint2 *dst, const uint8_t *__restrict__ smp,
                              const uint8_t *__restrict__ msk, int H, int W, int y0, int x0)
{
    const bool al = (W & 3) == 0 && (((uintptr_t)smp | (uintptr_t)msk) & 3) == 0;
    for (int i = threadIdx.x; i < RS * NWD; i += NT) {
        const int r = i / NWD, w = i - r * NWD;
        const int gy = y0 - HC + r, gx = x0 - HC + 4 * w;
        uint32_t vs = 0, vm = 0;
        if (gy >= 0 && gy < H) {
            const size_t ro = (size_t)gy * W;
            if (al && gx >= 0 && gx + 4 <= W) {          // one aligned word per plane
                vs = *reinterpret_cast<const uint32_t *>(smp + ro + gx);
                vm = *reinterpret_cast<const uint32_t *>(msk + ro + gx);
            } else {
                // 16-bit loads: W and gx are even, so a pixel pair never straddles the border
#pragma unroll
                for (int b = 0; b < 4; b += 2) {
                    const int x = gx + b;
                    if (x >= 0 && x < W) {
                        vs |= (uint32_t)(*reinterpret_cast<const uint16_t *>(smp + ro + x)) << (8 * b);
                        vm |= (uint32_t)(*reinterpret_cast<const uint16_t *>(msk + ro + x)) << (8 * b);
                    }
                }
            }
        }
        dst[r * RWDC + w] = make_uint2(vs, vm);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * RS * (NWD - 1); i += NT) {
        const int j = 1 + i / (RS * (NWD - 1));
        const int rem = i - (j - 1) * RS * (NWD - 1);
        const int r = rem / (NWD - 1), w = rem - r * (NWD - 1);
        const uint2 a = dst[r * RWDC + w], b = dst[r * RWDC + w + 1];
        dst[j * CPYC + r * RWDC + w] = make_uint2(__funnelshift_r(a.x, b.x, 8 * j),
                                                  __funnelshift_r(a.y, b.y, 8 * j));
    }
}

// acc + sum over the four bytes of |a - b|, one SIMD-video instruction with its accumulate
__device__ __forceinline__ int sad4_acc(uint32_t a, uint32_t b, int acc)
{
    int d;
    asm("vabsdiff4.u32.u32.u32.add %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(acc));
    return d;
}

// SAD over the measured current pixels of the T x T template whose top-left corner is at region
// (sy, sx), against the past-frame patch words P held in registers
template <int T>
__device__ __forceinline__ int sad_against(const Smem &sm, int sy, int sx, const uint32_t (&P)[T][3])
{
    constexpr uint32_t w0 = T >= 4 ? 0xffffffffu : (1u << (8 * T)) - 1u;
    constexpr uint32_t w1 = T >= 8 ? 0xffffffffu : (T > 4 ? (1u << (8 * (T - 4))) - 1u : 0u);
    constexpr uint32_t w2 = T >= 12 ? 0xffffffffu : (T > 8 ? (1u << (8 * (T - 8))) - 1u : 0u);
    const int j = sx & 3, w = sx >> 2;
    int acc = 0, acc1 = 0, acc2 = 0;          // one chain per template word: shorter latency
#pragma unroll
    for (int r = 0; r < T; ++r) {
        const uint2 *c = sm.csm + j * CPYC + (sy + r) * RWDC + w;
        const uint2 c0 = c[0];
        acc = sad4_acc(c0.x & w0, P[r][0] & c0.y & w0, acc);
        if (w1) {
            const uint2 c1 = c[1];
            acc1 = sad4_acc(c1.x & w1, P[r][1] & c1.y & w1, acc1);
        }
        if (w2) {
            const uint2 c2 = c[2];
            acc2 = sad4_acc(c2.x & w2, P[r][2] & c2.y & w2, acc2);
        }
    }
    return acc + acc1 + acc2;
}

// first past-frame word of this lane's rows r0 - 4 .. (F_d's second operand, independent of d)
__device__ __forceinline__ const uint32_t *box_ref(const Smem &sm, int r0, int wi, int vy, int vx)
{
    const int jr = (HC - 4 + vx) & 3, wr = wi + ((HC - 4 + vx) >> 2);
    return sm.rf + jr * CPY + (r0 - 4 + HC + vy) * RWD + wr;
}
// Box sums of F_d over the tile for one candidate d (T = 9).  F_d(y) = b_t(y + d) |s_t(y + d) -
// rec(y + v)| for tile rows r0 - 4 .. r0 + rows + 3 and the 4 columns 4 wi - 4 .. 4 wi - 1 of
// this lane (wi = 0 and 9 are the halo words), kept as vertical 9-sums in two packed 16-bit words
// (columns 0, 2 and 1, 3); the horizontal 9-sums come from the neighbouring lanes (lanes lane - 1
// and lane + 1 hold words wi - 1 and wi + 1) as in the forward ME.  refw(i) gives the past-frame
// word of row r0 - 4 + i; fn(j, h02, h13) receives the window sums (H0, H2) and (H1, H3) of
// output row r0 + j.
template <int ROWS, typename RefFn, typename Fn>
__device__ __forceinline__ void box_rows_ref(const Smem &sm, int r0, int wi, int dy, int dx, RefFn &&refw,
                                             Fn &&fn)
{
    const int jc = (HC - 4 + dx) & 3, wc = wi + ((HC - 4 + dx) >> 2);
    const uint2 *cur = sm.csm + jc * CPYC + (r0 - 4 + HC + dy) * RWDC + wc;
    uint32_t dlo[ROWS + 8], dhi[ROWS + 8], lo = 0, hi = 0;
#pragma unroll
    for (int i = 0; i < ROWS + 8; ++i) {
        const uint2 c = cur[i * RWDC];
        const uint32_t d4 = __vabsdiffu4(c.x, refw(i)) & c.y;
        dlo[i] = __byte_perm(d4, 0u, 0x4240);
        dhi[i] = __byte_perm(d4, 0u, 0x4341);
        lo += dlo[i];
        hi += dhi[i];
        if (i >= 9) {
            lo -= dlo[i - 9];
            hi -= dhi[i - 9];
        }
        if (i >= 8) {
            const uint32_t Q = lo + hi;
            const uint32_t Ql = __shfl_up_sync(0xffffffffu, Q, 1);
            const uint32_t lol = __shfl_up_sync(0xffffffffu, lo, 1);
            const uint32_t Qr = __shfl_down_sync(0xffffffffu, Q, 1);
            const uint32_t lor = __shfl_down_sync(0xffffffffu, lo, 1);
            const uint32_t A = __byte_perm(Ql, Q, 0x5432), B = __byte_perm(Q, Qr, 0x5432);
            const uint32_t h02 = Ql + A + Q + B + lor;
            fn(i - 8, h02, h02 + Qr - lol - lor);
        }
    }
}
template <int ROWS, typename Fn>
__device__ __forceinline__ void box_rows(const Smem &sm, int r0, int wi, int dy, int dx, int vy,
                                         int vx, Fn &&fn)
{
    const uint32_t *ref = box_ref(sm, r0, wi, vy, vx);
    box_rows_ref<ROWS>(sm, r0, wi, dy, dx, [&](int i) { return ref[i * RWD]; }, fn);
}

// FRMC reverse checks by box sums for the listed pixels whose filtered vector is v (T = 9).  The
// cost of candidate d at pixel p is C(p + d, v - d) = sum over o of F_d(p + o), a 9 x 9 box sum of
// one plane per candidate: the same integers the per-pixel path adds up, so the decisions are
// identical.  First each warp computes the d = 0 costs of 4 tile rows (lanes 0..9 hold the words)
// and stores them with the template counts, while the listed pixels with vector v are collected;
// then warp w takes candidates 1 + w, 9 + w, ... over the whole tile (lane = 3 chunks of 11 rows x
// 10 words), writes the candidate's cost at every tile pixel to its own plane, and compares only
// the collected pixels (at most a third of the unmeasured pixels of a tile are projectable, so a
// quarter of the tile or less): lane l keeps the verdicts of entries l, l + 32, ... as bits.
// They are merged over the warps and written to sm.rej for those pixels.
__device__ void box_checks9(Smem &sm, const FrameTask &t, int x0, int y0, int vy, int vx,
                            bool use_nnc)
{
    const int H = t.H, W = t.W, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool inner = y0 - kMaxRadius >= 0 && x0 - kMaxRadius >= 0 && y0 + TP + kMaxRadius <= H &&
                       x0 + TP + kMaxRadius <= W;
    {   // d = 0: rows 4 warp .. 4 warp + 3
        const int wi = min(lane, 9);
        box_rows<4>(sm, 4 * warp, wi, 0, 0, vy, vx, [&](int j, uint32_t h02, uint32_t h13) {
            if (lane >= 1 && lane <= 8) {
                const int r = 4 * warp + j, x = 4 * (wi - 1);
                const uint8_t *nr = &sm.nsrc[r + kMaxRadius][x + kMaxRadius];
                *reinterpret_cast<uint4 *>(&sm.e0n0[r][x]) =
                    make_uint4((h02 & 0xffffu) | (uint32_t)nr[0] << 16,
                               (h13 & 0xffffu) | (uint32_t)nr[1] << 16,
                               (h02 >> 16) | (uint32_t)nr[2] << 16, (h13 >> 16) | (uint32_t)nr[3] << 16);
            }
        });
        if (tid < 32) sm.rejb[tid] = 0;
        const int nl = sm.nlist;
        for (int li = tid; li < nl; li += NT) {
            const int pi = sm.list[li], py = pi / TP, px = pi - py * TP;
            const uint32_t c = use_nnc ? sm.md[py + 1][px + 1] : sm.mv[py + 2][px + 2];
            if (mv_y(c) == vy && mv_x(c) == vx) sm.blist[atomicAdd(&sm.nblist, 1)] = (uint16_t)pi;
            else plist(sm)[atomicAdd(&sm.nplist, 1)] = (uint16_t)pi;
        }
    }
    __syncthreads();
    const int nb = sm.nblist;
    for (int e = tid; e < nb; e += NT) {             // per-entry copies for the compares below
        const int pi = sm.blist[e], py = pi / TP, px = pi - py * TP;
        sm.be0n0[e] = sm.e0n0[py][px];
        sm.bnoff[e] = (uint16_t)((py + kMaxRadius) * NS + px + kMaxRadius);
    }
    __syncthreads();
    const int ch = min(lane / 10, 2), wi = lane < 30 ? lane - 10 * ch : 9;
    const bool out = lane < 30 && wi >= 1 && wi <= 8;
    uint32_t rej = 0;                                // bit i: entry lane + 32 i rejected
    const uint16_t *ec = &sm.ecand[warp][0][0];
    const uint8_t *ns = &sm.nsrc[0][0];
    // instantiated for interior tiles (every source p + d in the frame) and for the others
    // the past-frame words of the lane's rows are the same for every candidate d (the patch
    // around q = p + v stays fixed): loaded once, kept in registers (-3 % at 1080p)
    uint32_t refc[11 + 8];
    {
        const uint32_t *ref = box_ref(sm, 11 * ch, wi, vy, vx);
#pragma unroll
        for (int i = 0; i < 11 + 8; ++i) refc[i] = ref[i * RWD];
    }
    auto candidates = [&](auto inner_tag) {
        constexpr bool INNER = decltype(inner_tag)::value;
        for (int i = 1 + warp; i < 49; i += NW) {
            const int ci = i <= 24 ? i - 1 : i;      // the 48 offsets d != 0
            const int dy = frmc_offset(ci / 7), dx = frmc_offset(ci % 7);
            box_rows_ref<11>(sm, 11 * ch, wi, dy, dx, [&](int i) { return refc[i]; },
                             [&](int j, uint32_t h02, uint32_t h13) {
                const int r = 11 * ch + j;
                if (out && r < TP)                   // (H0, H1, H2, H3) of columns 4 (wi - 1) ..
                    *reinterpret_cast<uint2 *>(&sm.ecand[warp][r][4 * (wi - 1)]) =
                        make_uint2(__byte_perm(h02, h13, 0x5410), __byte_perm(h02, h13, 0x7632));
            });
            __syncwarp();
            const int doff = dy * NS + dx;
#pragma unroll 4
            for (int e = lane, b = 0; e < nb; e += 32, ++b) {
                const int pi = sm.blist[e];
                bool valid = true;
                if constexpr (!INNER) {
                    const int py = pi / TP, px = pi - py * TP;
                    valid = (unsigned)(y0 + py + dy) < (unsigned)H && (unsigned)(x0 + px + dx) < (unsigned)W;
                }
                const uint32_t z = sm.be0n0[e];
                const int ev = ec[pi];
                const int nr = ns[sm.bnoff[e] + doff];
                if (valid && ev * (int)(z >> 16) < (int)(z & 0xffffu) * nr) rej |= 1u << b;
            }
            __syncwarp();                            // the plane is rewritten by the next candidate
        }
    };
    if (inner) candidates(std::true_type{});
    else candidates(std::false_type{});
    if (rej) atomicOr(&sm.rejb[lane], rej);
    __syncthreads();
    for (int e = tid; e < nb; e += NT) sm.rej[sm.blist[e]] = (sm.rejb[e & 31] >> (e >> 5)) & 1u;
}

__device__ __forceinline__ void cp4(void *dst, const void *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// asynchronous copies of past frame k's ME field (rows y0-2 .. y0+33, columns x0-2 .. x0+33) and,
// for the reverse checks, of the past frame (rows y0-HC .., words from column x0-HC) into the raw
// buffers; the caller checked that both regions lie inside the frame and are 4-byte aligned
__device__ void prefetch_past(Smem &sm, const FrameTask &t, int k, int x0, int y0, bool rf)
{
    const int W = t.W;
    const uint8_t *mv = reinterpret_cast<const uint8_t *>(t.mv[k]);
    for (int i = threadIdx.x; i < MT * MT / 2; i += NT) {
        const int r = i / (MT / 2), w = i - r * (MT / 2);
        cp4(&sm.mvraw[i], mv + ((size_t)(y0 - 2 + r) * W + (x0 - 2)) * 2 + 4 * w);
    }
    if (rf) {
        const uint8_t *ref = t.ref_rec[k];
        for (int i = threadIdx.x; i < RS * NWD; i += NT) {
            const int r = i / NWD, w = i - r * NWD;
            cp4(&sm.rfraw[i], ref + (size_t)(y0 - HC + r) * W + (x0 - HC) + 4 * w);
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int T>
__device__ __forceinline__ void cc_tile(Smem &sm, const FrameTask &t, int tbx, int tby)
{
    constexpr int h = T / 2;
    const int H = t.H, W = t.W;
    const int x0 = tbx * TP, y0 = tby * TP;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (*t.status) return;
    const bool use_nnc = t.cc_mode == 4 || t.cc_mode == 5;
    const bool frmc = t.cc_mode == 3 || t.cc_mode == 5;
    const bool rmc = t.cc_mode == 2;
    const bool rme = t.cc_mode == 1;

    // interior tiles of 4-byte aligned planes fetch each past frame's ME field and past frame
    // with cp.async while the previous one is checked (-4 % at 1080p: the loads' latency no
    // longer sits between the checks of consecutive past frames)
    bool pf = (W & 3) == 0 && y0 >= HC && x0 >= HC && y0 + TP + HC <= H && x0 + 4 * NWD - HC <= W;
    for (int k = 0; k < t.K; ++k)
        pf = pf && (((uintptr_t)t.mv[k] | (uintptr_t)t.ref_rec[k]) & 3) == 0;
    if (pf && t.K > 0) prefetch_past(sm, t, 0, x0, y0, frmc || rmc);
    if (frmc || rmc) {
        const uint4 *src = reinterpret_cast<const uint4 *>(&g_order[frmc ? 0 : t.Rc]);
        uint4 *dst = reinterpret_cast<uint4 *>(&sm.ord);
        for (int i = tid; i < (int)(sizeof(CandOrder) / sizeof(uint4)); i += NT) dst[i] = src[i];
    }
    stage_current(sm.csm, t.cur_smp, t.cur_msk, H, W, y0, x0);
    __syncthreads();
    // template counts n around every source position of the tile +- 9 (current mask, 0 outside),
    // separably: T-column counts of every staged row the sources need, then T-row sums of those
    {
        constexpr int HR = NS + T - 1;                     // staged rows the sources' templates span
        static_assert(HR * NS <= (int)sizeof(sm.e0n0), "row counts fit the box-check buffer");
        uint8_t *hc = reinterpret_cast<uint8_t *>(sm.e0n0);   // unused until the checks
        for (int i = tid; i < HR * NS; i += NT) {
            const int r = i / NS, sx = i - r * NS;
            const int ry = r + HC - kMaxRadius - h, rx = sx + HC - kMaxRadius - h;
            const uint2 *cm = sm.csm + (rx & 3) * CPYC + ry * RWDC + (rx >> 2);
            int n = 0;
#pragma unroll
            for (int b = 0; b < (T + 3) / 4; ++b) {
                uint32_t m = cm[b].y;
                if (4 * b + 4 > T) m &= (1u << (8 * (T - 4 * b))) - 1u;
                n += __popc(m);
            }
            hc[i] = (uint8_t)(n >> 3);
        }
        __syncthreads();
        for (int i = tid; i < NS * NS; i += NT) {
            const int sy = i / NS, sx = i - sy * NS;
            int n = 0;
#pragma unroll
            for (int r = 0; r < T; ++r) n += hc[(sy + r) * NS + sx];
            sm.nsrc[sy][sx] = (uint8_t)n;
        }
    }

    int sum[PPT], cnt[PPT];
#pragma unroll
    for (int i = 0; i < PPT; ++i) sum[i] = cnt[i] = 0;

    for (int k = 0; k < t.K; ++k) {
        const uint16_t *mvk = reinterpret_cast<const uint16_t *>(t.mv[k]);   // (v_y, v_x) bytes
        if (pf) cp_wait_all();
        __syncthreads();
        if (pf) {
            for (int i = tid; i < MT * MT; i += NT) {
                const int r = i / MT, c = i - r * MT;
                sm.mv[r][c] = pack_mv(sm.mvraw[r * (MT / 2) + (c >> 1)], c & 1);
            }
            if (frmc || rmc)
                for (int i = tid; i < RS * NWD; i += NT) {
                    const int r = i / NWD, w = i - r * NWD;
                    sm.rf[r * RWD + w] = sm.rfraw[i];
                }
        } else {
            for (int i = tid; i < MT * MT; i += NT) {
                const int r = i / MT, c = i - r * MT;
                const int gy = min(max(y0 - 2 + r, 0), H - 1), gx = min(max(x0 - 2 + c, 0), W - 1);
                sm.mv[r][c] = pack_mv(mvk[(size_t)gy * W + gx], 0);
            }
            if (frmc || rmc) stage_past0(sm.rf, t.ref_rec[k], H, W, y0, x0);
        }
        if (tid == 0) sm.nlist = sm.nblist = sm.nplist = 0;
        __syncthreads();
        if (pf && k + 1 < t.K) prefetch_past(sm, t, k + 1, x0, y0, frmc || rmc);   // buffers read
        if (frmc || rmc) shift_past(sm.rf);
        if (use_nnc) {
            // in the same phase as the shifted copies (it reads only the staged field): a thread
            // slides along MSEG medians of one row, each sorted column serving three of them
            for (int i = tid; i < MD * MNSEG; i += NT) {
                const int r = i / MNSEG, c0 = (i - r * MNSEG) * MSEG;
                auto col = [&](int c) { return psort3(sm.mv[r][c], sm.mv[r + 1][c], sm.mv[r + 2][c]); };
                Sorted3 a = col(c0), b = col(c0 + 1);
#pragma unroll
                for (int j = 0; j < MSEG; ++j) {
                    if (c0 + j >= MD) break;
                    const Sorted3 c = col(c0 + j + 2);
                    sm.md[r][c0 + j] = pmedian9(a, b, c);
                    a = b;
                    b = c;
                }
            }
        }
        if constexpr (T == 9) {                 // vector histogram of the listed pixels (below)
            if (frmc)
                for (int i = tid; i < HS * HS; i += NT) sm.hist[i] = 0;
        }
        __syncthreads();
        // decide every pixel; list the ones that need a reverse check.  First the filtered vector,
        // the NNC verdict and q = p + v of all pixels of the thread, with the loads of the past
        // mask at q (and of the reverse field in RME mode) issued together; then the decisions.
        uint8_t dec[PPT];
        int qv[PPT];
        uint32_t fv[PPT];
        bool pass[PPT], meas[PPT], pend[PPT];
        uint8_t qm[PPT];
        char2 rw[PPT];
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
            const int pi = tid + i * NT, py = pi / TP, px = pi - py * TP;
            const int y = y0 + py, x = x0 + px;
            qv[i] = -1;
            pend[i] = false;
            pass[i] = true;
            meas[i] = false;
            qm[i] = 0;
            if (y >= H || x >= W) continue;
            uint32_t c;
            if (use_nnc) {
                c = sm.md[py + 1][px + 1];
                const int nb[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int yy = y + nb[j][0], xx = x + nb[j][1];
                    if ((unsigned)yy >= (unsigned)H || (unsigned)xx >= (unsigned)W) continue;
                    if (!near1(c, sm.md[py + 1 + nb[j][0]][px + 1 + nb[j][1]])) pass[i] = false;
                }
            } else {
                c = sm.mv[py + 2][px + 2];
            }
            fv[i] = c;
            const int fy = mv_y(c), fx = mv_x(c);
            const size_t gi = (size_t)y * W + x;
            reinterpret_cast<char2 *>(t.fmv[k])[gi] = make_char2((signed char)fy, (signed char)fx);
            const int qy = y + fy, qx = x + fx;
            const uint32_t mword = sm.csm[(py + HC) * RWDC + ((px + HC) >> 2)].y;
            meas[i] = ((mword >> (8 * ((px + HC) & 3))) & 0xffu) != 0;
            if (!meas[i] && (unsigned)qy < (unsigned)H && (unsigned)qx < (unsigned)W) {
                qv[i] = qy * W + qx;
                qm[i] = t.ref_msk[k][qv[i]];
                if (rme) rw[i] = reinterpret_cast<const char2 *>(t.rmv[k])[qv[i]];
            }
        }
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
            const int pi = tid + i * NT, py = pi / TP, px = pi - py * TP;
            dec[i] = 255;
            if (y0 + py >= H || x0 + px >= W) continue;
            if (meas[i]) {
                dec[i] = 0;
            } else if (qv[i] < 0 || !qm[i]) {
                dec[i] = 1;
                qv[i] = -1;
            } else if (use_nnc && !pass[i]) {
                dec[i] = 2;
            } else if (rme) {
                dec[i] = (rw[i].x == -mv_y(fv[i]) && rw[i].y == -mv_x(fv[i])) ? 4 : 3;
            } else if (frmc || rmc) {
                dec[i] = 254;                                   // pending reverse check
                pend[i] = true;
            } else {
                dec[i] = 4;
            }
        }
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
            if (!pend[i]) continue;
            const int pi = tid + i * NT;
            sm.rej[pi] = 0;
            sm.list[atomicAdd(&sm.nlist, 1)] = (uint16_t)pi;
            if constexpr (T == 9) {
                if (frmc) atomicAdd(&sm.hist[(mv_y(fv[i]) + kMaxRadius) * HS + mv_x(fv[i]) + kMaxRadius], 1);
            }
        }
        __syncthreads();
        const int nl = sm.nlist;
        // FRMC, T = 9: box-sum checks for the vector that most listed pixels share, if at least
        // BOX_MIN do.  The cost of a candidate over the whole tile is one box sum, so the 49
        // candidates cost about as much as 70 per-pixel checks.  Under quarter sampling at most a
        // third of the unmeasured pixels of a tile are projectable per past frame (256), so one
        // vector pays for it in most tiles.  RMC stays per pixel: its 289 candidates make the box
        // pass dearer than per-pixel checks, which stop at the first better candidate.
        int boxbin = -1;
        if constexpr (T == 9) {
            if (frmc && nl >= BOX_MIN) {
                if (warp == 0) {                                  // the most frequent bin
                    uint32_t key = 0;                              // count << 10 | 1023 - bin
                    for (int i = lane; i < HS * HS; i += 32)
                        key = max(key, ((uint32_t)sm.hist[i] << 10) | (1023u - i));
                    key = __reduce_max_sync(0xffffffffu, key);
                    if (lane == 0) sm.boxv = (int)(key >> 10) >= BOX_MIN ? 1023 - (int)(key & 1023u) : -1;
                }
                __syncthreads();                                  // before plist overwrites hist
                boxbin = sm.boxv;
                if (boxbin >= 0)
                    box_checks9(sm, t, x0, y0, boxbin / HS - kMaxRadius, boxbin % HS - kMaxRadius,
                                use_nnc);
            }
        }
        // reverse checks of the other listed pixels: one warp per pixel
        const uint16_t *pl = boxbin >= 0 ? plist(sm) : sm.list;
        const int np = boxbin >= 0 ? sm.nplist : nl;
        for (int li = warp; li < np; li += NW) {
            const int pi = pl[li], py = pi / TP, px = pi - py * TP;
            const uint32_t c = use_nnc ? sm.md[py + 1][px + 1] : sm.mv[py + 2][px + 2];
            const int fy = mv_y(c), fx = mv_x(c);
            uint32_t P[T][3];                          // past-frame patch around q
            {
                const int ry = py + HC + fy - h, rx = px + HC + fx - h;
                const uint32_t *base = sm.rf + (rx & 3) * CPY + ry * RWD + (rx >> 2);
#pragma unroll
                for (int r = 0; r < T; ++r) {
                    P[r][0] = base[r * RWD];
                    P[r][1] = base[r * RWD + 1];
                    P[r][2] = base[r * RWD + 2];
                }
            }
            // candidate of round rd of this lane: its cost, template count and validity
            const int ph = (px + HC - h) & 3;
            auto score = [&](int rd, int &s, int &n) {
                const int e = sm.ord.lane[ph][rd][lane];
                s = n = 0;
                if (e == NOCAND) return false;
                const int dy = cand_dy(e, frmc, t.Rc), dx = cand_dx(e, frmc, t.Rc);
                const int sy = y0 + py + dy, sx = x0 + px + dx;
                if ((unsigned)sy >= (unsigned)H || (unsigned)sx >= (unsigned)W) return false;
                s = sad_against<T>(sm, py + dy + HC - h, px + dx + HC - h, P);
                n = sm.nsrc[py + dy + kMaxRadius][px + dx + kMaxRadius];
                return true;
            };
            bool rej = false;
            const int nround = sm.ord.nround[ph];
            if (frmc) {
                // FRMC fills two rounds (49 candidates): both are scored in one pass, so that
                // their shared-memory loads and SAD chains overlap
                int s0, n0, s1, n1;
                bool v0 = score(0, s0, n0);
                const bool v1 = score(1, s1, n1);
                const int sc = __shfl_sync(0xffffffffu, s0, 0), nc = __shfl_sync(0xffffffffu, n0, 0);
                if (lane == 0) v0 = false;                  // round 0, lane 0 scores d = 0
                const bool better = (v0 && s0 * nc < sc * n0) || (v1 && s1 * nc < sc * n1);
                rej = __any_sync(0xffffffffu, better);
            } else {
                int sc = 0, nc = 0;
                for (int rd = 0; rd < nround; ++rd) {
                    int s, n;
                    bool valid = score(rd, s, n);
                    if (rd == 0) {
                        sc = __shfl_sync(0xffffffffu, s, 0);
                        nc = __shfl_sync(0xffffffffu, n, 0);
                        if (lane == 0) valid = false;
                    }
                    const bool better = valid && s * nc < sc * n;
                    if (__any_sync(0xffffffffu, better)) {
                        rej = true;
                        break;
                    }
                }
            }
            if (lane == 0) sm.rej[pi] = rej ? 1 : 0;
        }
        __syncthreads();
        const uint8_t *rs = t.ref_smp[k];
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
            if (dec[i] == 255) continue;
            const int pi = tid + i * NT, py = pi / TP, px = pi - py * TP;
            uint8_t d = dec[i];
            if (d == 254) d = sm.rej[pi] ? 3 : 4;
            t.dec[k][(size_t)(y0 + py) * W + x0 + px] = d;
            if (d == 4) {
                sum[i] += rs[qv[i]];
                cnt[i] += 1;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
        const int pi = tid + i * NT, py = pi / TP, px = pi - py * TP;
        const int y = y0 + py, x = x0 + px;
        if (y >= H || x >= W) continue;
        t.psum[(size_t)y * W + x] = (uint16_t)sum[i];
        t.pcnt[(size_t)y * W + x] = (uint8_t)cnt[i];
    }
}

// template cost at a single source (RME reverse field): SAD over measured current pixels
__device__ void cost_at(const FrameTask &t, const uint8_t *__restrict__ ref, int sy, int sx,
                        int vy, int vx, int &sad, int &n)
{
    const int h = t.T / 2, H = t.H, W = t.W;
    int s = 0, c = 0;
    for (int oy = -h; oy <= h; ++oy) {
        const int y = sy + oy;
        if ((unsigned)y >= (unsigned)H) continue;
        const int ry = min(max(y + vy, 0), H - 1);
        const uint8_t *crow = t.cur_smp + (size_t)y * W;
        const uint8_t *mrow = t.cur_msk + (size_t)y * W;
        const uint8_t *rrow = ref + (size_t)ry * W;
        for (int ox = -h; ox <= h; ++ox) {
            const int x = sx + ox;
            if ((unsigned)x >= (unsigned)W || !mrow[x]) continue;
            const int rx = min(max(x + vx, 0), W - 1);
            s += iabs((int)crow[x] - (int)rrow[rx]);
            c += 1;
        }
    }
    sad = s;
    n = c;
}

__device__ __forceinline__ bool tie_before(int ay, int ax, int by, int bx)
{
    const int la = iabs(ay) + iabs(ax), lb = iabs(by) + iabs(bx);
    if (la != lb) return la < lb;
    if (ay != by) return ay < by;
    return ax < bx;
}

template <int T>
__global__ void __launch_bounds__(NT) cc_project_kernel(FrameTask t)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cc_tile<T>(*reinterpret_cast<Smem *>(smem_raw), t, blockIdx.x, blockIdx.y);
}

template <int T>
__global__ void __launch_bounds__(NT) cc_batched_kernel(BatchDesc *bd)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ FrameTask task;
    __shared__ int claim[2];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    claim_tiles(bd, kPhCc, task, claim, [&](const FrameTask &t, int l) {
        const int tx = (t.W + TP - 1) / TP;
        cc_tile<T>(sm, t, l % tx, l / tx);
    });
}

// ---------------------------------------------------------------------------------------------
// Fused ME + checks + projection (T = 9): one persistent launch per frame.  The CTAs (8 warps,
// the checks' shared memory, which also holds an ME strip's staging) claim items in order from a
// host-built list: ME tiles of 64-row bands (me9_tile with 8 warp strips) and check tiles.  An ME
// tile ends with a barrier and a release increment of its band's counter; a check tile first
// waits (one thread, bounded polls with back-off) until the bands it reads -- rows y0 - 2 ..
// y0 + 33 for the median halo -- are complete, then every thread acquires the counters itself
// before reading the motion fields.  Items are claimed one at a time and every item's
// dependencies come earlier in the list, so the lowest unfinished item can always proceed.  A
// wait that runs out marks the frame (kStatusWaitTimeout) and later tiles skip their work.
// ---------------------------------------------------------------------------------------------
constexpr int F_MEW = 8;                          // warps of an ME item (64-row strips)
constexpr int F_MEROWS = me9k::s_outh<F_MEW>();
static_assert(sizeof(me9k::Smem9<F_MEW>) <= sizeof(Smem), "an ME strip's staging fits the checks' smem");
static_assert(me9k::s_nt<F_MEW>() == NT, "ME items use every thread of the CTA");

// item: bit 31 check tile (else ME tile), bits 0..9 tile column, 10..21 tile row, 22..23 past frame
constexpr uint32_t F_CC = 0x80000000u;
__host__ __device__ constexpr uint32_t f_item(bool cc, int tx, int ty, int k)
{
    return (cc ? F_CC : 0u) | (uint32_t)tx | ((uint32_t)ty << 10) | ((uint32_t)k << 22);
}
// ME bands lo..hi that check-tile row ty reads (rows 32 ty - 2 .. 32 ty + 33)
__host__ __device__ constexpr int f_band_lo(int ty) { return ty == 0 ? 0 : (TP * ty - 2) / F_MEROWS; }
__host__ __device__ constexpr int f_band_hi(int ty, int nbands)
{
    return (TP * ty + TP + 1) / F_MEROWS < nbands - 1 ? (TP * ty + TP + 1) / F_MEROWS : nbands - 1;
}

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// t.status points at a word of m.ctr that stays 0 during the launch: the tiles test it on entry,
// and a status that another CTA could change meanwhile might split a CTA at its barriers.
// The frame's own status word is m.status.
__global__ void __launch_bounds__(NT, 2) mecc_kernel(FrameTask t, MeccPlan m)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    me9k::Smem9<F_MEW> &sm9 = *reinterpret_cast<me9k::Smem9<F_MEW> *>(smem_raw);
    __shared__ int claim, failed, skip;
    if (threadIdx.x == 0) skip = *(volatile int *)m.status;   // bad mask: nothing to do, nothing waits
    __syncthreads();
    if (skip) return;                             // uniform over the CTA
    for (;;) {
        if (threadIdx.x == 0) claim = atomicAdd(&m.ctr[0], 1);
        __syncthreads();
        const int i = claim;
        if (i >= m.nitems) break;                 // uniform over the CTA
        const uint32_t it = m.items[i];
        const int tx = (int)(it & 0x3ffu), ty = (int)((it >> 10) & 0xfffu), k = (int)((it >> 22) & 3u);
        if (!(it & F_CC)) {
            me9k::me9_tile<F_MEW>(sm9, t, tx, ty, k);
            __syncthreads();                      // every motion vector of the tile is written
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(&m.ctr[2 + ty], 1);
            }
        } else {
            const int lo = f_band_lo(ty), hi = f_band_hi(ty, m.nbands);
            if (threadIdx.x == 0) {
                int bad = ld_acquire(&m.ctr[1]);
                for (int b = lo; b <= hi && !bad; ++b) {
                    int n = 0;
                    while (ld_acquire(&m.ctr[2 + b]) < m.need + m.bias) {
                        if (++n > m.limit) {
                            bad = 1;
                            break;
                        }
                        __nanosleep(256);
                    }
                }
                if (bad) {
                    atomicExch(&m.ctr[1], 1);
                    atomicOr(m.status, kStatusWaitTimeout);
                }
                failed = bad;
            }
            __syncthreads();
            if (!failed) {
                for (int b = lo; b <= hi; ++b) (void)ld_acquire(&m.ctr[2 + b]);   // this thread's acquire
                cc_tile<9>(sm, t, tx, ty);
                cp_wait_all();                    // no copy into shared memory outlives the tile
            }
        }
        __syncthreads();                          // the claim slot and shared memory are reused
    }
}

// RME (Sec. 2.2): reverse motion vector at every past-frame pixel q: argmin over w in [-R, R]^2
// with q + w inside of C(q + w, -w), exact mean-cost order, tie order on w.
__device__ __forceinline__ void rme_tile(const FrameTask &t, int tbx, int tby, int k)
{
    const int qx = tbx * 32 + (threadIdx.x & 31);
    const int qy = tby * (NT / 32) + (threadIdx.x >> 5);
    if (qx >= t.W || qy >= t.H || *t.status) return;
    const int R = t.R;
    int bs = 0, bn = 0, by = 0, bx = 0;
    bool have = false;
    for (int wy = -R; wy <= R; ++wy) {
        const int sy = qy + wy;
        if ((unsigned)sy >= (unsigned)t.H) continue;
        for (int wx = -R; wx <= R; ++wx) {
            const int sx = qx + wx;
            if ((unsigned)sx >= (unsigned)t.W) continue;
            int s, n;
            cost_at(t, t.ref_rec[k], sy, sx, -wy, -wx, s, n);
            const long long l = (long long)s * bn, r = (long long)bs * n;
            if (!have || l < r || (l == r && tie_before(wy, wx, by, bx))) {
                bs = s; bn = n; by = wy; bx = wx; have = true;
            }
        }
    }
    reinterpret_cast<char2 *>(t.rmv[k])[(size_t)qy * t.W + qx] =
        make_char2((signed char)by, (signed char)bx);
}

__global__ void __launch_bounds__(NT) rme_field_kernel(FrameTask t)
{
    rme_tile(t, blockIdx.x, blockIdx.y, blockIdx.z);
}

__global__ void __launch_bounds__(NT) rme_batched_kernel(BatchDesc *bd)
{
    __shared__ FrameTask task;
    __shared__ int claim[2];
    claim_tiles(bd, kPhRme, task, claim, [](const FrameTask &t, int l) {
        const int tx = (t.W + 31) / 32, ty = (t.H + NT / 32 - 1) / (NT / 32);
        rme_tile(t, l % tx, (l / tx) % ty, l / (tx * ty));
    });
}

int g_order_ready[64];

// The dynamic shared-memory limit of a kernel is a per-device attribute: set it once on every
// device the kernel is launched on (done[d] per device ordinal d).
template <typename K>
cudaError_t set_smem(K kernel, std::atomic<bool> (&done)[64])
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (done[dev].load()) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
    if (e == cudaSuccess) done[dev].store(true);
    return e;
}

template <int T>
cudaError_t launch_cc_t(const FrameTask &t, cudaStream_t st)
{
    static std::atomic<bool> attr[64];
    cudaError_t e = set_smem(cc_project_kernel<T>, attr);
    if (e != cudaSuccess) return e;
    dim3 grid((t.W + TP - 1) / TP, (t.H + TP - 1) / TP);
    cc_project_kernel<T><<<grid, NT, sizeof(Smem), st>>>(t);
    return cudaGetLastError();
}

template <int T>
cudaError_t launch_cc_batched_t(BatchDesc *bd, cudaStream_t st)
{
    static std::atomic<bool> attr[64];
    cudaError_t e = set_smem(cc_batched_kernel<T>, attr);
    if (e != cudaSuccess) return e;
    static std::atomic<int> grids[64];
    const int grid = persistent_grid_cached(cc_batched_kernel<T>, NT, sizeof(Smem), grids);
    cc_batched_kernel<T><<<grid, NT, sizeof(Smem), st>>>(bd);
    return cudaGetLastError();
}

}  // namespace

int tiles_cc(const FrameTask &t) { return ((t.W + TP - 1) / TP) * ((t.H + TP - 1) / TP); }

int mecc_bands(int H) { return (H + F_MEROWS - 1) / F_MEROWS; }
int mecc_need(int W, int K) { return ((W + me9k::S_OUTW - 1) / me9k::S_OUTW) * K; }

// Claim order: the ME bands top to bottom (every column tile and past frame of a band), and each
// check-tile row once the band holding its last needed row is `lag` bands back, lag being about
// one wave of the grid, so that a check tile is normally claimed after its bands are done.
int mecc_schedule(int H, int W, int K, int grid, uint32_t *items)
{
    const int nb = mecc_bands(H), nc = (W + me9k::S_OUTW - 1) / me9k::S_OUTW;
    const int ny = (H + TP - 1) / TP, nx = (W + TP - 1) / TP;
    const int per_band = std::max(1, nc * K);
    const int lag = (grid + per_band - 1) / per_band + 1;
    int n = 0, row = 0;
    auto emit_rows = [&](int upto_band) {
        while (row < ny && f_band_hi(row, nb) <= upto_band) {
            for (int x = 0; x < nx; ++x, ++n)
                if (items) items[n] = f_item(true, x, row, 0);
            ++row;
        }
    };
    for (int b = 0; b < nb; ++b) {
        for (int k = 0; k < K; ++k)
            for (int c = 0; c < nc; ++c, ++n)
                if (items) items[n] = f_item(false, c, b, k);
        emit_rows(b - lag);
    }
    emit_rows(nb);
    return n;
}

// the shared-memory attribute comes first: the occupancy query counts on it
static std::atomic<bool> g_mecc_attr[64];
int mecc_grid()
{
    if (set_smem(mecc_kernel, g_mecc_attr) != cudaSuccess) return 0;
    static std::atomic<int> grids[64];
    return persistent_grid_cached(mecc_kernel, NT, sizeof(Smem), grids);
}

cudaError_t launch_me_cc(const FrameTask &t, const MeccPlan &plan, cudaStream_t st)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = init_cc(dev);
    if (e != cudaSuccess) return e;
    const int grid = mecc_grid();
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    mecc_kernel<<<grid, NT, sizeof(Smem), st>>>(t, plan);
    count_launch();
    return cudaGetLastError();
}

cudaError_t init_cc(int dev)
{
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (g_order_ready[dev]) return cudaSuccess;
    struct Orders {
        CandOrder o[NORDER];
        bool ok;
    };
    static const Orders *host = [] {            // built once (thread-safe static initialisation)
        auto *r = new Orders();
        r->ok = true;
        for (int i = 0; i < NORDER; ++i) {
            build_order(r->o[i], i == 0, i);
            r->ok = r->ok && order_ok(r->o[i], i == 0, i);
        }
        return r;
    }();
    if (!host->ok) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemcpyToSymbol(g_order, host->o, sizeof(host->o));
    if (e == cudaSuccess) g_order_ready[dev] = 1;
    return e;
}

int tiles_rme(const FrameTask &t)
{
    if (t.K <= 0 || t.cc_mode != 1) return 0;
    if (t.T == 9) return tiles_rme9(t);
    return ((t.W + 31) / 32) * ((t.H + NT / 32 - 1) / (NT / 32)) * t.K;
}

cudaError_t launch_cc_project(const FrameTask &t, cudaStream_t st)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = init_cc(dev);
    if (e != cudaSuccess) return e;
    switch (t.T) {
    case 1: e = launch_cc_t<1>(t, st); break;
    case 3: e = launch_cc_t<3>(t, st); break;
    case 5: e = launch_cc_t<5>(t, st); break;
    case 7: e = launch_cc_t<7>(t, st); break;
    case 9: e = launch_cc_t<9>(t, st); break;
    case 11: e = launch_cc_t<11>(t, st); break;
    default: return cudaErrorInvalidValue;
    }
    count_launch();
    return e;
}

cudaError_t launch_cc_batched(BatchDesc *bd, int T, cudaStream_t st)
{
    cudaError_t e;
    switch (T) {
    case 1: e = launch_cc_batched_t<1>(bd, st); break;
    case 3: e = launch_cc_batched_t<3>(bd, st); break;
    case 5: e = launch_cc_batched_t<5>(bd, st); break;
    case 7: e = launch_cc_batched_t<7>(bd, st); break;
    case 9: e = launch_cc_batched_t<9>(bd, st); break;
    case 11: e = launch_cc_batched_t<11>(bd, st); break;
    default: return cudaErrorInvalidValue;
    }
    count_launch();
    return e;
}

cudaError_t launch_rme_field(const FrameTask &t, cudaStream_t st)
{
    if (t.K <= 0) return cudaSuccess;
    if (t.T == 9) return launch_rme9(t, st);
    dim3 grid((t.W + 31) / 32, (t.H + NT / 32 - 1) / (NT / 32), t.K);
    rme_field_kernel<<<grid, NT, 0, st>>>(t);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_rme_batched(BatchDesc *bd, int T, cudaStream_t st)
{
    if (T == 9) return launch_rme9_batched(bd, st);
    static std::atomic<int> grids[64];
    const int grid = persistent_grid_cached(rme_batched_kernel, NT, 0, grids);
    rme_batched_kernel<<<grid, NT, 0, st>>>(bd);
    count_launch();
    return cudaGetLastError();
}

}  // namespace rfsr
