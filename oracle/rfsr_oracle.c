/*
 * rfsr_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow CPU restatement of the per-frame hot path of recursive
 * frequency-selective reconstruction of quarter-sampled video (Grosche, Seiler, Kaup,
 * "Novel Consistency Check for Fast Recursive Reconstruction of Non-Regularly Sampled Video
 * Data", ICIP 2021, arXiv 2203.09200).  Only the tests, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load it.  It shares no code, header, table or
 * constant generator with the CUDA library; the two only share the seeded input generators.
 *
 * What it computes, in the paper's order (Fig. 1 flow: ME -> CC -> PR -> FSR):
 *   orc_cost ........ template-matching cost of Sec. 2.2 (masked SAD over a T x T template of the
 *                     current frame's measured pixels against a reconstructed past frame)
 *   orc_me_pixel .... pixel-wise motion estimation of Sec. 2.2 (argmin over the search window)
 *   orc_me_pixel_predictive  the opt-in predictive-centre search (not in the paper)
 *   orc_nnc_field ... nearest neighbour check, Sec. 3.1.2 and Eq. (1)
 *   orc_check_* ..... reverse motion estimation RME (Sec. 2.2), reverse motion check RMC and fast
 *                     reverse motion check FRMC (Sec. 3.1.1, Fig. 2b/2c)
 *   orc_cc_project .. combination of the checks (Sec. 3.1.2: NNC first, FRMC only for survivors)
 *                     and projection of measured past pixels with averaging (Sec. 2.2)
 *   orc_fsr_block ... block-wise frequency selective reconstruction (Sec. 2.1) with the D-FSR
 *                     overwrite rule of Sec. 3.2 and concealed weighting zero (Sec. 4)
 *   orc_quantize .... 8-bit reconstruction that becomes the next frame's reference
 *
 * Built plainly it is single-threaded.  Built with -fopenmp (a second library), the frame-level
 * loops over pixels and blocks -- each of which writes only its own outputs -- run on several
 * threads; the arithmetic and the results are the same.
 *
 * The paper leaves several details open.  The readings taken here (the cost function, the tie
 * order, border handling, the FSR model and its constants) are listed in the design notes and
 * repeated at each function.  Parity status: every function is pinned by tests/test_oracle_*.py
 * against closed forms, invariants, library routines or brute force; the FSR constants (rho,
 * gamma, frequency weighting, iteration count) are not given by the paper and are configuration,
 * so FSR parity against the paper itself is limited to those structural pins.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_VERSION 1

/* threads of the OpenMP build (no effect in the single-threaded build) */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

/* decision labels per pixel and reference frame */
enum { DEC_MEASURED = 0, DEC_NOT_PROJECTABLE = 1, DEC_NNC_REJECT = 2, DEC_CHECK_REJECT = 3,
       DEC_ACCEPT = 4 };
/* consistency check modes (Table 3 rows plus "none" and NNC alone) */
enum { CC_NONE = 0, CC_RME = 1, CC_RMC = 2, CC_FRMC = 3, CC_NNC = 4, CC_NNC_FRMC = 5 };

int orc_version(void) { return ORC_VERSION; }

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }
static int iabs(int v) { return v < 0 ? -v : v; }
static int inside(int y, int x, int H, int W) { return y >= 0 && y < H && x >= 0 && x < W; }

/* ---------------------------------------------------------------------------------------------
 * Sec. 2.2: pixel-wise template matching between the measured data of the current frame and an
 * already reconstructed past frame.  Reading: the template is the T x T window around p; only
 * pixels measured in the current frame (mask 1, inside the frame) contribute; the cost is the sum
 * of absolute differences against the past frame at the same offsets displaced by v, with past
 * frame coordinates clamped to the border.  n counts the contributing pixels.
 * ------------------------------------------------------------------------------------------- */
void orc_cost(const uint8_t *smp, const uint8_t *msk, const uint8_t *ref, int H, int W, int T,
              int py, int px, int vy, int vx, int *sad_out, int *n_out)
{
    int h = T / 2, sad = 0, n = 0;
    for (int oy = -h; oy <= h; ++oy) {
        for (int ox = -h; ox <= h; ++ox) {
            int y = py + oy, x = px + ox;
            if (!inside(y, x, H, W) || !msk[(size_t)y * W + x]) continue;
            int ry = clampi(y + vy, 0, H - 1), rx = clampi(x + vx, 0, W - 1);
            sad += iabs((int)smp[(size_t)y * W + x] - (int)ref[(size_t)ry * W + rx]);
            n += 1;
        }
    }
    *sad_out = sad;
    *n_out = n;
}

/* Tie order between two displacement vectors (the paper states none): smaller |y|+|x| first,
 * then smaller y, then smaller x.  Returns 1 if a comes strictly before b. */
static int tie_before(int ay, int ax, int by, int bx)
{
    int la = iabs(ay) + iabs(ax), lb = iabs(by) + iabs(bx);
    if (la != lb) return la < lb;
    if (ay != by) return ay < by;
    return ax < bx;
}

/* Candidate a = (sad_a, n_a, vector a) is strictly better than b: costs are compared as the mean
 * absolute difference sad/n (exactly, by cross multiplication); equal means fall back to the tie
 * order.  For forward motion estimation n does not depend on v, so this is the plain SAD order. */
int orc_better(int sad_a, int n_a, int ay, int ax, int sad_b, int n_b, int by, int bx)
{
    long long l = (long long)sad_a * n_b, r = (long long)sad_b * n_a;
    if (l != r) return l < r;
    return tie_before(ay, ax, by, bx);
}

/* Sec. 2.2: motion vector of pixel p into the past frame: argmin of the template cost over
 * v in [-R, R]^2 with p + v inside the frame. */
void orc_me_pixel(const uint8_t *smp, const uint8_t *msk, const uint8_t *ref, int H, int W,
                  int T, int R, int py, int px, int8_t *vy_out, int8_t *vx_out)
{
    int bs = 0, bn = 0, by = 0, bx = 0, have = 0;
    for (int vy = -R; vy <= R; ++vy) {
        for (int vx = -R; vx <= R; ++vx) {
            if (!inside(py + vy, px + vx, H, W)) continue;
            int s, n;
            orc_cost(smp, msk, ref, H, W, T, py, px, vy, vx, &s, &n);
            if (!have || orc_better(s, n, vy, vx, bs, bn, by, bx)) {
                bs = s; bn = n; by = vy; bx = vx; have = 1;
            }
        }
    }
    *vy_out = (int8_t)by;
    *vx_out = (int8_t)bx;
}

/* Dense motion vector field (alpha, beta) of Sec. 3.1.2: one vector per pixel, stored as
 * mv[2*(y*W+x)] = vertical component, mv[2*(y*W+x)+1] = horizontal component. */
void orc_me_field(const uint8_t *smp, const uint8_t *msk, const uint8_t *ref, int H, int W,
                  int T, int R, int8_t *mv)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            orc_me_pixel(smp, msk, ref, H, W, T, R, y, x, &mv[2 * ((size_t)y * W + x)],
                         &mv[2 * ((size_t)y * W + x) + 1]);
}

/* Predictive-centre search, an opt-in variant that the paper does not describe (it changes the
 * method's results): past frame t-k, k >= 2, is searched only within radius Rp of the prediction
 * k v1(p), where v1 is the full-search vector of p to frame t-1.  The prediction is clamped into
 * [-R, R]^2 and so that p + c lies in the frame; the candidates are the v of c + [-Rp, Rp]^2 that
 * lie in [-R, R]^2 with p + v in the frame, ranked by the same cost and tie order as
 * orc_me_pixel.  k is the past frame's distance (2 for t-2). */
void orc_me_pixel_predictive(const uint8_t *smp, const uint8_t *msk, const uint8_t *ref, int H,
                             int W, int T, int R, int Rp, int k, int v1y, int v1x, int py, int px,
                             int8_t *vy_out, int8_t *vx_out)
{
    int cy = clampi(k * v1y, -R > -py ? -R : -py, R < H - 1 - py ? R : H - 1 - py);
    int cx = clampi(k * v1x, -R > -px ? -R : -px, R < W - 1 - px ? R : W - 1 - px);
    int bs = 0, bn = 0, by = 0, bx = 0, have = 0;
    for (int vy = cy - Rp; vy <= cy + Rp; ++vy) {
        for (int vx = cx - Rp; vx <= cx + Rp; ++vx) {
            if (iabs(vy) > R || iabs(vx) > R || !inside(py + vy, px + vx, H, W)) continue;
            int s, n;
            orc_cost(smp, msk, ref, H, W, T, py, px, vy, vx, &s, &n);
            if (!have || orc_better(s, n, vy, vx, bs, bn, by, bx)) {
                bs = s; bn = n; by = vy; bx = vx; have = 1;
            }
        }
    }
    *vy_out = (int8_t)by;
    *vx_out = (int8_t)bx;
}

/* the predictive field of past frame t-k from the field mv1 of t-1 (same layout as mv) */
void orc_me_field_predictive(const uint8_t *smp, const uint8_t *msk, const uint8_t *ref, int H,
                             int W, int T, int R, int Rp, int k, const int8_t *mv1, int8_t *mv)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t i = 2 * ((size_t)y * W + x);
            orc_me_pixel_predictive(smp, msk, ref, H, W, T, R, Rp, k, mv1[i], mv1[i + 1], y, x,
                                    &mv[i], &mv[i + 1]);
        }
}

/* ---------------------------------------------------------------------------------------------
 * Eq. (1), Sec. 3.1.2: component-wise 3x3 median of the vector field (border replicated), then
 * for every pixel the filtered vectors of the four nearest neighbours (m-1,n), (m+1,n), (m,n-1),
 * (m,n+1) that lie inside the frame are compared with the pixel's own filtered vector; the vector
 * passes iff every such pair differs by at most one in the sum of absolute component differences.
 * ------------------------------------------------------------------------------------------- */
static int median9(int *a)
{
    for (int i = 1; i < 9; ++i) {        /* insertion sort of nine values */
        int v = a[i], j = i - 1;
        while (j >= 0 && a[j] > v) { a[j + 1] = a[j]; --j; }
        a[j + 1] = v;
    }
    return a[4];
}

static void median_vector(const int8_t *mv, int H, int W, int y, int x, int *my, int *mx)
{
    int ay[9], ax[9], c = 0;
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            int yy = clampi(y + dy, 0, H - 1), xx = clampi(x + dx, 0, W - 1);
            ay[c] = mv[2 * ((size_t)yy * W + xx)];
            ax[c] = mv[2 * ((size_t)yy * W + xx) + 1];
            ++c;
        }
    *my = median9(ay);
    *mx = median9(ax);
}

void orc_nnc_field(const int8_t *mv, int H, int W, int8_t *fmv, uint8_t *pass)
{
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int my, mx;
            median_vector(mv, H, W, y, x, &my, &mx);
            fmv[2 * ((size_t)y * W + x)] = (int8_t)my;
            fmv[2 * ((size_t)y * W + x) + 1] = (int8_t)mx;
        }
    static const int NB[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int ok = 1;
            int cy = fmv[2 * ((size_t)y * W + x)], cx = fmv[2 * ((size_t)y * W + x) + 1];
            for (int i = 0; i < 4; ++i) {
                int yy = y + NB[i][0], xx = x + NB[i][1];
                if (!inside(yy, xx, H, W)) continue;
                int ny = fmv[2 * ((size_t)yy * W + xx)], nx = fmv[2 * ((size_t)yy * W + xx) + 1];
                if (iabs(cy - ny) + iabs(cx - nx) > 1) ok = 0;
            }
            pass[(size_t)y * W + x] = (uint8_t)ok;
        }
}

/* ---------------------------------------------------------------------------------------------
 * Reverse checks.  For a pixel p with (filtered) vector v, let q = p + v in the past frame.  A
 * reverse vector w from q into the current frame is scored with the same template cost, taken
 * with its template centred at the current-frame source position q + w and the past frame
 * displaced by -w, i.e. cost(q + w, -w): the patch of the past frame around q stays fixed and the
 * current-frame template slides.  Sources outside the frame are not candidates.
 * ------------------------------------------------------------------------------------------- */

/* Sec. 3.1.1 (Fig. 2b, 2c): RMC tests the reverse vectors -v + d for every d in [-Rc, Rc]^2;
 * FRMC tests only d with both components in {-7,-3,-1,0,1,3,7}.  The vector is accepted iff the
 * reverse vector pointing back to p (d = 0) has the lowest cost; d = 0 comes first in the tie
 * order, so it wins ties. */
static const int FRMC_SET[7] = {-7, -3, -1, 0, 1, 3, 7};

static int reverse_check(const uint8_t *smp, const uint8_t *msk, const uint8_t *ref, int H,
                         int W, int T, int py, int px, int vy, int vx, const int *set, int nset)
{
    int s0, n0;
    orc_cost(smp, msk, ref, H, W, T, py, px, vy, vx, &s0, &n0);   /* d = 0: cost(p, v) */
    for (int i = 0; i < nset; ++i)
        for (int j = 0; j < nset; ++j) {
            int dy = set[i], dx = set[j];
            if (dy == 0 && dx == 0) continue;
            int sy = py + dy, sx = px + dx;                         /* source p + d = q + w */
            if (!inside(sy, sx, H, W)) continue;
            int s, n;
            orc_cost(smp, msk, ref, H, W, T, sy, sx, vy - dy, vx - dx, &s, &n);
            if (orc_better(s, n, dy, dx, s0, n0, 0, 0)) return 0;
        }
    return 1;
}

int orc_check_frmc(const uint8_t *smp, const uint8_t *msk, const uint8_t *ref, int H, int W,
                   int T, int py, int px, int vy, int vx)
{
    return reverse_check(smp, msk, ref, H, W, T, py, px, vy, vx, FRMC_SET, 7);
}

int orc_check_rmc(const uint8_t *smp, const uint8_t *msk, const uint8_t *ref, int H, int W,
                  int T, int Rc, int py, int px, int vy, int vx)
{
    int set[64], n = 0;
    for (int d = -Rc; d <= Rc; ++d) set[n++] = d;
    return reverse_check(smp, msk, ref, H, W, T, py, px, vy, vx, set, n);
}

/* Sec. 2.2 (RME of the literature method): the full reverse motion estimation at q: argmin over
 * w in [-R, R]^2 with q + w inside the frame of cost(q + w, -w), tie order applied to w. */
void orc_rme_vector(const uint8_t *smp, const uint8_t *msk, const uint8_t *ref, int H, int W,
                    int T, int R, int qy, int qx, int8_t *wy_out, int8_t *wx_out)
{
    int bs = 0, bn = 0, by = 0, bx = 0, have = 0;
    for (int wy = -R; wy <= R; ++wy)
        for (int wx = -R; wx <= R; ++wx) {
            int sy = qy + wy, sx = qx + wx;
            if (!inside(sy, sx, H, W)) continue;
            int s, n;
            orc_cost(smp, msk, ref, H, W, T, sy, sx, -wy, -wx, &s, &n);
            if (!have || orc_better(s, n, wy, wx, bs, bn, by, bx)) {
                bs = s; bn = n; by = wy; bx = wx; have = 1;
            }
        }
    *wy_out = (int8_t)by;
    *wx_out = (int8_t)bx;
}

/* RME accepts iff both vectors coincide: the reverse vector found at q points back to p. */
int orc_check_rme(const uint8_t *smp, const uint8_t *msk, const uint8_t *ref, int H, int W,
                  int T, int R, int py, int px, int vy, int vx)
{
    int8_t wy, wx;
    orc_rme_vector(smp, msk, ref, H, W, T, R, py + vy, px + vx, &wy, &wx);
    return wy == -vy && wx == -vx;
}

/* ---------------------------------------------------------------------------------------------
 * Checks + projection for one past frame (Sec. 2.2 projection, Sec. 3.1.2 combination).
 * For each pixel p of the current frame, in this order:
 *   measured in the current frame                    -> DEC_MEASURED (nothing to project)
 *   q = p + v outside the frame or not measured in
 *   the past frame (only measurements are projected) -> DEC_NOT_PROJECTABLE
 *   NNC mode and the NNC fails                        -> DEC_NNC_REJECT
 *   RME / RMC / FRMC mode and the check fails         -> DEC_CHECK_REJECT
 *   otherwise                                         -> DEC_ACCEPT: psum += past sample at q,
 *                                                        pcnt += 1
 * v is the median-filtered vector when the mode includes NNC and the raw vector otherwise.
 * The projected value of a pixel is psum / pcnt, the average over the past frames that project
 * (Sec. 2.2).  fmv receives the vector used, dec the labels.
 * ------------------------------------------------------------------------------------------- */
void orc_cc_project(int cc_mode, int T, int R, int Rc, const uint8_t *smp, const uint8_t *msk,
                    const uint8_t *ref_rec, const uint8_t *ref_smp, const uint8_t *ref_msk,
                    int H, int W, const int8_t *mv, int8_t *fmv, uint8_t *dec, uint16_t *psum,
                    uint8_t *pcnt)
{
    int use_nnc = (cc_mode == CC_NNC || cc_mode == CC_NNC_FRMC);
    uint8_t *pass = (uint8_t *)malloc((size_t)H * W);
    if (use_nnc) {
        orc_nnc_field(mv, H, W, fmv, pass);
    } else {
        memcpy(fmv, mv, (size_t)H * W * 2);
        memset(pass, 1, (size_t)H * W);
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t i = (size_t)y * W + x;
            int vy = fmv[2 * i], vx = fmv[2 * i + 1];
            int qy = y + vy, qx = x + vx;
            uint8_t d;
            if (msk[i]) d = DEC_MEASURED;
            else if (!inside(qy, qx, H, W) || !ref_msk[(size_t)qy * W + qx]) d = DEC_NOT_PROJECTABLE;
            else if (use_nnc && !pass[i]) d = DEC_NNC_REJECT;
            else {
                int ok = 1;
                if (cc_mode == CC_FRMC || cc_mode == CC_NNC_FRMC)
                    ok = orc_check_frmc(smp, msk, ref_rec, H, W, T, y, x, vy, vx);
                else if (cc_mode == CC_RMC)
                    ok = orc_check_rmc(smp, msk, ref_rec, H, W, T, Rc, y, x, vy, vx);
                else if (cc_mode == CC_RME)
                    ok = orc_check_rme(smp, msk, ref_rec, H, W, T, R, y, x, vy, vx);
                d = ok ? DEC_ACCEPT : DEC_CHECK_REJECT;
            }
            dec[i] = d;
            if (d == DEC_ACCEPT) {
                psum[i] = (uint16_t)(psum[i] + ref_smp[(size_t)qy * W + qx]);
                pcnt[i] = (uint8_t)(pcnt[i] + 1);
            }
        }
    free(pass);
}

/* The same decision for a single pixel, computing only the vectors it needs (its own and, for
 * the NNC modes, those of the 3x3 windows around it and its four neighbours).  Used to check
 * sampled pixels of full-size frames. */
static void me_vec_at(const uint8_t *smp, const uint8_t *msk, const uint8_t *ref, int H, int W,
                      int T, int R, int y, int x, int *vy, int *vx)
{
    int8_t a, b;
    orc_me_pixel(smp, msk, ref, H, W, T, R, clampi(y, 0, H - 1), clampi(x, 0, W - 1), &a, &b);
    *vy = a;
    *vx = b;
}

static void median_at(const uint8_t *smp, const uint8_t *msk, const uint8_t *ref, int H, int W,
                      int T, int R, int y, int x, int *my, int *mx)
{
    int ay[9], ax[9], c = 0;
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            me_vec_at(smp, msk, ref, H, W, T, R, clampi(y + dy, 0, H - 1),
                      clampi(x + dx, 0, W - 1), &ay[c], &ax[c]);
            ++c;
        }
    *my = median9(ay);
    *mx = median9(ax);
}

int orc_cc_pixel(int cc_mode, int T, int R, int Rc, const uint8_t *smp, const uint8_t *msk,
                 const uint8_t *ref_rec, const uint8_t *ref_smp, const uint8_t *ref_msk,
                 int H, int W, int y, int x, int8_t *mv_out, int8_t *fmv_out, int *proj_val)
{
    int use_nnc = (cc_mode == CC_NNC || cc_mode == CC_NNC_FRMC);
    int vy, vx, fy, fx, pass = 1;
    me_vec_at(smp, msk, ref_rec, H, W, T, R, y, x, &vy, &vx);
    if (use_nnc) {
        static const int NB[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};
        median_at(smp, msk, ref_rec, H, W, T, R, y, x, &fy, &fx);
        for (int i = 0; i < 4; ++i) {
            int yy = y + NB[i][0], xx = x + NB[i][1];
            if (!inside(yy, xx, H, W)) continue;
            int ny, nx;
            median_at(smp, msk, ref_rec, H, W, T, R, yy, xx, &ny, &nx);
            if (iabs(fy - ny) + iabs(fx - nx) > 1) pass = 0;
        }
    } else {
        fy = vy;
        fx = vx;
    }
    mv_out[0] = (int8_t)vy; mv_out[1] = (int8_t)vx;
    fmv_out[0] = (int8_t)fy; fmv_out[1] = (int8_t)fx;
    *proj_val = -1;
    size_t i = (size_t)y * W + x;
    int qy = y + fy, qx = x + fx;
    if (msk[i]) return DEC_MEASURED;
    if (!inside(qy, qx, H, W) || !ref_msk[(size_t)qy * W + qx]) return DEC_NOT_PROJECTABLE;
    if (use_nnc && !pass) return DEC_NNC_REJECT;
    int ok = 1;
    if (cc_mode == CC_FRMC || cc_mode == CC_NNC_FRMC)
        ok = orc_check_frmc(smp, msk, ref_rec, H, W, T, y, x, fy, fx);
    else if (cc_mode == CC_RMC)
        ok = orc_check_rmc(smp, msk, ref_rec, H, W, T, Rc, y, x, fy, fx);
    else if (cc_mode == CC_RME)
        ok = orc_check_rme(smp, msk, ref_rec, H, W, T, R, y, x, fy, fx);
    if (!ok) return DEC_CHECK_REJECT;
    *proj_val = ref_smp[(size_t)qy * W + qx];
    return DEC_ACCEPT;
}

/* ---------------------------------------------------------------------------------------------
 * Frequency selective reconstruction (Sec. 2.1) of one B x B block from its N x N support, with
 * the projected pixels of Sec. 2.2 used as additional known pixels "in the same manner" as the
 * measured ones and the D-FSR overwrite rule of Sec. 3.2.  Concealed weighting is zero (Sec. 4),
 * so each block depends only on measured / projected pixels and all blocks are independent.
 *
 * The paper defers the model to the single-frame FSR of its reference [Seiler 2015]; the reading
 * used here is the standard FSR matching-pursuit loop with a real-valued model kept as conjugate
 * pairs of DFT basis functions:
 *   support coordinates (m, n) in [0, N)^2, frame pixel (B*by - o + m, B*bx - o + n), o = (N-B)/2
 *   known pixel: measured (f = s/255, weight rho^d) or projected (f = psum/(255*pcnt), weight
 *   mu*rho^d); d = distance to the support centre ((N-1)/2, (N-1)/2); other pixels weight 0
 *   W(k,l) = DFT of the weights, R(k,l) = DFT of weight*(f - g), g = 0 at the start
 *   each iteration: u = canonical bin of a conjugate pair maximising wf(u) |R(u)|^2 (ties to the
 *     lowest linear index k*N+l); dc = gamma R(u) / W(0,0);
 *     model g += dc phi_u + conj(dc) phi_-u   (self-conjugate u: g += Re(dc) phi_u)
 *     R(k) -= dc W(k-u) + conj(dc) W(k+u)     (self-conjugate u: R(k) -= Re(dc) W(k-u))
 *   wf(k,l) = (1 - sqrt(2)/2 * sqrt(kn^2 + ln^2))^2 with kn = min(k, N-k)/(N/2), likewise ln
 *   output: g at the block pixels, replaced by s/255 where measured (D-FSR; the R-FSR flag also
 *   replaces projected pixels by their projected value).
 * phi_u(m,n) = exp(2 pi i (u_k m + u_l n) / N); the DFT uses exp(-2 pi i (k m + l n) / N).
 * ------------------------------------------------------------------------------------------- */
typedef struct {
    int B;              /* block size */
    int N;              /* support size = DFT size */
    int iterations;     /* number of model iterations */
    double rho;         /* spatial weighting decay */
    double gamma;       /* orthogonality deficiency compensation */
    double proj_weight; /* weight factor of projected pixels (1: same manner as measured) */
    int overwrite_projected; /* 0: D-FSR (measured only overwrite), 1: R-FSR */
} orc_fsr_params;

#define ORC_NMAX 64

static double freq_weight(int k, int l, int N)
{
    double kn = (double)(k < N - k ? k : N - k) / (N / 2.0);
    double ln = (double)(l < N - l ? l : N - l) / (N / 2.0);
    double t = 1.0 - sqrt(2.0) / 2.0 * sqrt(kn * kn + ln * ln);
    return t * t;
}

/* cos / sin of 2 pi j / N for j = 0..N-1 (angles of the N-point DFT). */
static void twiddles(int N, double *c, double *s)
{
    for (int j = 0; j < N; ++j) {
        c[j] = cos(2.0 * M_PI * j / N);
        s[j] = sin(2.0 * M_PI * j / N);
    }
}

/* 2-D DFT of a real N x N array a (row-major), as two passes of 1-D DFTs (along n, then m):
 * X(k,l) = sum_m sum_n a(m,n) exp(-2 pi i (k m + l n) / N). */
static void dft2_real(const double *a, int N, const double *tc, const double *ts, double *re,
                      double *im)
{
    static _Thread_local double tr[ORC_NMAX * ORC_NMAX], ti[ORC_NMAX * ORC_NMAX];
    for (int m = 0; m < N; ++m)
        for (int l = 0; l < N; ++l) {
            double sr = 0.0, si = 0.0;
            for (int n = 0; n < N; ++n) {
                int j = (l * n) % N;                 /* exp(-i a) = cos a - i sin a */
                sr += a[m * N + n] * tc[j];
                si -= a[m * N + n] * ts[j];
            }
            tr[m * N + l] = sr;
            ti[m * N + l] = si;
        }
    for (int k = 0; k < N; ++k)
        for (int l = 0; l < N; ++l) {
            double sr = 0.0, si = 0.0;
            for (int m = 0; m < N; ++m) {
                int j = (k * m) % N;
                double c = tc[j], s = -ts[j];
                sr += tr[m * N + l] * c - ti[m * N + l] * s;
                si += tr[m * N + l] * s + ti[m * N + l] * c;
            }
            re[k * N + l] = sr;
            im[k * N + l] = si;
        }
}

/* The N x N support of block (by, bx) (Sec. 2.1): known pixels are the measured ones (value
 * s/255, weight rho^d, d = distance to the support centre) and the projected ones (value
 * psum / (255 pcnt), weight proj_weight rho^d); with concealed weighting delta > 0 (the original
 * FSR, which the paper sets to zero in Sec. 4 so that blocks are independent), the pixels of
 * blocks already reconstructed in raster order that are neither measured nor projected are known
 * too, with value conc (their reconstruction) and weight delta rho^d.  Everything else, and
 * everything outside the frame, has weight 0. */
static void fsr_support(const orc_fsr_params *P, double delta, const double *conc,
                        const uint8_t *smp, const uint8_t *msk, const uint16_t *psum,
                        const uint8_t *pcnt, int H, int W, int by, int bx, double *w, double *f)
{
    const int N = P->N, B = P->B, o = (P->N - P->B) / 2;
    const double c = (N - 1) / 2.0;
    for (int m = 0; m < N; ++m)
        for (int n = 0; n < N; ++n) {
            int y = B * by - o + m, x = B * bx - o + n;
            double d = sqrt((m - c) * (m - c) + (n - c) * (n - c));
            double wt = 0.0, val = 0.0;
            if (inside(y, x, H, W)) {
                size_t i = (size_t)y * W + x;
                int earlier = y / B < by || (y / B == by && x / B < bx);
                if (msk[i]) { wt = pow(P->rho, d); val = smp[i] / 255.0; }
                else if (pcnt && pcnt[i] > 0) {
                    wt = P->proj_weight * pow(P->rho, d);
                    val = (double)psum[i] / (255.0 * pcnt[i]);
                } else if (conc && delta > 0.0 && earlier) {
                    wt = delta * pow(P->rho, d);
                    val = conc[i];
                }
            }
            w[m * N + n] = wt;
            f[m * N + n] = val;
        }
}

/* Outcome of a replay (fsr_block_core with a followed selection sequence). */
typedef struct {
    int iterations_run;   /* iterations taken; the followed sequence may end early (0xffff)      */
    int divergences;      /* iterations whose followed pair is not this evaluation's argmax      */
    int first_div;        /* the first such iteration, -1 if none                                 */
    int invalid;          /* 1: a followed index is not the canonical member of a pair          */
    double first_gap;     /* (best - followed) / best criterion at the first divergence          */
    double max_gap;       /* the largest such relative gap over all divergences (0 if none)      */
    double max_scale;     /* at that divergence: 2 S / |R(best)|, S = max_k |R_0(k)| plus
                             2 gamma sum_j |R(u_j)| over the earlier iterations -- the magnitude
                             that the rounding of the residual's arithmetic scales with          */
    double max_excess;    /* max over divergences of gap / (bound_q + bound_u * 2 S / |R(best)|),
                             for a caller-given bound of that form (0 if none is given)          */
} orc_fsr_replay;

#define ORC_SEL_NONE 0xffffu   /* a followed entry meaning "no further iteration" */

/* Extended form for tests: besides the B*B block output it can return the support weights and
 * values, the model g over the whole support, the final residual spectrum, the selected bins, the
 * relative gap between the best and second best selection criterion at every iteration and their
 * minimum.
 * Replay: with follow != NULL, iteration i updates the model with the pair follow[i] instead of
 * its own argmax (and stops at the first ORC_SEL_NONE).  Sec. 2.1's update is a function of the
 * selected pair, so following the selections another evaluation of the same method made (an FP32
 * one, say) gives that evaluation's result up to its rounding; rep records where and by how much
 * the followed pair's criterion fell short of this evaluation's maximum. */
static void fsr_block_core(const orc_fsr_params *P, double delta, const double *conc,
                           const uint8_t *smp, const uint8_t *msk, const uint16_t *psum,
                           const uint8_t *pcnt, int H, int W, int by, int bx, double *out,
                           double *w_out, double *f_out, double *g_out, double *rre_out,
                           double *rim_out, int *sel_out, double *min_gap_out, double *gaps_out,
                           const uint16_t *follow, const double *bound, orc_fsr_replay *rep)
{
    const int N = P->N, B = P->B, o = (P->N - P->B) / 2;
    static _Thread_local double w[ORC_NMAX * ORC_NMAX], f[ORC_NMAX * ORC_NMAX];
    static _Thread_local double wf[ORC_NMAX * ORC_NMAX];
    static _Thread_local double Wre[ORC_NMAX * ORC_NMAX], Wim[ORC_NMAX * ORC_NMAX];
    static _Thread_local double Rre[ORC_NMAX * ORC_NMAX], Rim[ORC_NMAX * ORC_NMAX];
    static _Thread_local double g[ORC_NMAX * ORC_NMAX], fw[ORC_NMAX * ORC_NMAX];
    static _Thread_local double tc[ORC_NMAX], ts[ORC_NMAX];
    twiddles(N, tc, ts);
    fsr_support(P, delta, conc, smp, msk, psum, pcnt, H, W, by, bx, w, f);
    for (int i = 0; i < N * N; ++i) {
        fw[i] = w[i] * f[i];
        g[i] = 0.0;
        wf[i] = freq_weight(i / N, i % N, N);
    }
    dft2_real(w, N, tc, ts, Wre, Wim);
    dft2_real(fw, N, tc, ts, Rre, Rim);

    double min_gap = INFINITY;
    const double W0 = Wre[0];
    orc_fsr_replay rp = {0, 0, -1, 0, 0.0, 0.0, 0.0, 0.0};
    double scale = 0.0;                       /* S of orc_fsr_replay */
    for (int i = 0; i < N * N; ++i) {
        double a = sqrt(Rre[i] * Rre[i] + Rim[i] * Rim[i]);
        if (a > scale) scale = a;
    }
    for (int it = 0; it < P->iterations && W0 > 0.0; ++it) {
        int best = -1, best2 = -1;
        double bv = -1.0, second = -1.0;
        for (int k = 0; k < N; ++k)
            for (int l = 0; l < N; ++l) {
                int lin = k * N + l, conj_lin = ((N - k) % N) * N + (N - l) % N;
                if (lin > conj_lin) continue;                 /* canonical member of the pair */
                double e = wf[lin] * (Rre[lin] * Rre[lin] + Rim[lin] * Rim[lin]);
                if (e > bv) { second = bv; best2 = best; bv = e; best = lin; }
                else if (e > second) { second = e; best2 = lin; }
            }
        double gap = (bv > 0.0 && second >= 0.0) ? (bv - second) / bv : INFINITY;
        if (gap < min_gap) min_gap = gap;
        if (gaps_out) gaps_out[it] = gap;
        (void)best2;
        if (follow) {
            unsigned fl = follow[it];
            if (fl == ORC_SEL_NONE) break;
            int fk = (int)fl / N, fc = (int)fl % N;
            if ((int)fl >= N * N || (int)fl > ((N - fk) % N) * N + (N - fc) % N) {
                rp.invalid = 1;
                break;
            }
            if ((int)fl != best) {
                double ef = wf[fl] * (Rre[fl] * Rre[fl] + Rim[fl] * Rim[fl]);
                double g = bv > 0.0 ? (bv - ef) / bv : 0.0;
                double rb = sqrt(Rre[best] * Rre[best] + Rim[best] * Rim[best]);
                if (rp.divergences == 0) { rp.first_div = it; rp.first_gap = g; }
                double sc = rb > 0.0 ? 2.0 * scale / rb : INFINITY;
                if (g > rp.max_gap) {
                    rp.max_gap = g;
                    rp.max_scale = sc;
                }
                if (bound) {
                    double x = g / (bound[0] + bound[1] * sc);
                    if (x > rp.max_excess) rp.max_excess = x;
                }
                rp.divergences++;
            }
            best = (int)fl;
        }
        scale += 2.0 * P->gamma * sqrt(Rre[best] * Rre[best] + Rim[best] * Rim[best]);
        rp.iterations_run = it + 1;
        int uk = best / N, ul = best % N;
        int self = (((N - uk) % N) == uk) && (((N - ul) % N) == ul);
        double dre = P->gamma * Rre[best] / W0, dim = P->gamma * Rim[best] / W0;
        if (self) dim = 0.0;
        if (sel_out) sel_out[it] = best;
        /* model update over the support */
        for (int m = 0; m < N; ++m)
            for (int n = 0; n < N; ++n) {
                int j = (uk * m + ul * n) % N;
                double re_part = dre * tc[j] - dim * ts[j];         /* Re(dc * phi_u) */
                g[m * N + n] += self ? re_part : 2.0 * re_part;
            }
        /* residual spectrum update */
        for (int k = 0; k < N; ++k)
            for (int l = 0; l < N; ++l) {
                int a = ((k - uk + N) % N) * N + (l - ul + N) % N;     /* W(k - u) */
                int b = ((k + uk) % N) * N + (l + ul) % N;             /* W(k + u) */
                double xr = dre * Wre[a] - dim * Wim[a];
                double xi = dre * Wim[a] + dim * Wre[a];
                if (!self) {                                            /* conj(dc) W(k + u) */
                    xr += dre * Wre[b] + dim * Wim[b];
                    xi += dre * Wim[b] - dim * Wre[b];
                }
                Rre[k * N + l] -= xr;
                Rim[k * N + l] -= xi;
            }
    }
    for (int m = 0; m < B; ++m)
        for (int n = 0; n < B; ++n) {
            int y = B * by + m, x = B * bx + n;
            double v = g[(o + m) * N + (o + n)];
            if (inside(y, x, H, W)) {
                size_t i = (size_t)y * W + x;
                if (msk[i]) v = smp[i] / 255.0;
                else if (P->overwrite_projected && pcnt && pcnt[i] > 0)
                    v = (double)psum[i] / (255.0 * pcnt[i]);
            }
            out[m * B + n] = v;
        }
    if (w_out) memcpy(w_out, w, sizeof(double) * N * N);
    if (f_out) memcpy(f_out, f, sizeof(double) * N * N);
    if (g_out) memcpy(g_out, g, sizeof(double) * N * N);
    if (rre_out) memcpy(rre_out, Rre, sizeof(double) * N * N);
    if (rim_out) memcpy(rim_out, Rim, sizeof(double) * N * N);
    if (min_gap_out) *min_gap_out = min_gap;
    if (rep) *rep = rp;
}

/* One block with every trace (support, model, final residual, selections, gaps), for the tests. */
void orc_fsr_block_ex(const orc_fsr_params *P, const uint8_t *smp, const uint8_t *msk,
                      const uint16_t *psum, const uint8_t *pcnt, int H, int W, int by, int bx,
                      double *out, double *w_out, double *f_out, double *g_out, double *rre_out,
                      double *rim_out, int *sel_out, double *min_gap_out, double *gaps_out)
{
    fsr_block_core(P, 0.0, NULL, smp, msk, psum, pcnt, H, W, by, bx, out, w_out, f_out, g_out,
                   rre_out, rim_out, sel_out, min_gap_out, gaps_out, NULL, NULL, NULL);
}

/* One block with concealed weighting delta and concealed values conc (H x W, may be NULL for
 * delta = 0), along its own argmax (follow = NULL) or along the selection sequence
 * follow[0 .. iterations) (replay, see fsr_block_core); sel_out, min_gap_out, gaps_out and rep
 * may be NULL. */
void orc_fsr_block_replay(const orc_fsr_params *P, double delta, const double *conc,
                          const uint8_t *smp, const uint8_t *msk, const uint16_t *psum,
                          const uint8_t *pcnt, int H, int W, int by, int bx,
                          const uint16_t *follow, const double *bound, double *out, int *sel_out,
                          double *min_gap_out, double *gaps_out, orc_fsr_replay *rep)
{
    fsr_block_core(P, delta, conc, smp, msk, psum, pcnt, H, W, by, bx, out, 0, 0, 0, 0, 0, sel_out,
                   min_gap_out, gaps_out, follow, bound, rep);
}

void orc_fsr_block(const orc_fsr_params *P, const uint8_t *smp, const uint8_t *msk,
                   const uint16_t *psum, const uint8_t *pcnt, int H, int W, int by, int bx,
                   double *out, double *min_gap_out)
{
    fsr_block_core(P, 0.0, NULL, smp, msk, psum, pcnt, H, W, by, bx, out, 0, 0, 0, 0, 0, 0,
                   min_gap_out, 0, NULL, NULL, NULL);
}

/* Every block of the frame; out is H x W (pixels of partial edge blocks outside the frame are
 * dropped), min_gap holds one value per block (row-major over blocks).  follow (may be NULL):
 * replay every block along its selection sequence, follow[b * iterations ..] for block b; rep
 * (may be NULL) then receives one record per block, with max_excess measured against
 * bound = {bound_q, bound_u} (may be NULL). */
void orc_fsr_frame_replay(const orc_fsr_params *P, const uint8_t *smp, const uint8_t *msk,
                          const uint16_t *psum, const uint8_t *pcnt, int H, int W,
                          const uint16_t *follow, const double *bound, double *out,
                          double *min_gap, orc_fsr_replay *rep)
{
    int B = P->B, nby = (H + B - 1) / B, nbx = (W + B - 1) / B;
#pragma omp parallel for schedule(dynamic, 1)
    for (int by = 0; by < nby; ++by)
        for (int bx = 0; bx < nbx; ++bx) {
            double blk[ORC_NMAX * ORC_NMAX];
            double gap;
            const int b = by * nbx + bx;
            fsr_block_core(P, 0.0, NULL, smp, msk, psum, pcnt, H, W, by, bx, blk, 0, 0, 0, 0, 0, 0,
                           &gap, 0, follow ? follow + (size_t)b * P->iterations : NULL, bound,
                           rep ? rep + b : NULL);
            if (min_gap) min_gap[b] = gap;
            for (int m = 0; m < B; ++m)
                for (int n = 0; n < B; ++n) {
                    int y = B * by + m, x = B * bx + n;
                    if (inside(y, x, H, W)) out[(size_t)y * W + x] = blk[m * B + n];
                }
        }
}

void orc_fsr_frame(const orc_fsr_params *P, const uint8_t *smp, const uint8_t *msk,
                   const uint16_t *psum, const uint8_t *pcnt, int H, int W, double *out,
                   double *min_gap)
{
    orc_fsr_frame_replay(P, smp, msk, psum, pcnt, H, W, NULL, NULL, out, min_gap, NULL);
}

/* FSR of every block with concealed weighting delta (the original FSR; the paper uses delta = 0,
 * Sec. 4): blocks are reconstructed one after the other in raster order, and each sees the pixels
 * of the blocks before it that are neither measured nor projected as known pixels with their
 * reconstruction as value and weight delta rho^d.  out (H x W) also serves as that input; the
 * result for delta = 0 equals orc_fsr_frame. */
void orc_fsr_frame_concealed(const orc_fsr_params *P, double delta, const uint8_t *smp,
                             const uint8_t *msk, const uint16_t *psum, const uint8_t *pcnt, int H,
                             int W, const uint16_t *follow, const double *bound, double *out,
                             double *min_gap, orc_fsr_replay *rep)
{
    int B = P->B, nby = (H + B - 1) / B, nbx = (W + B - 1) / B;
    memset(out, 0, sizeof(double) * (size_t)H * W);
    for (int by = 0; by < nby; ++by)
        for (int bx = 0; bx < nbx; ++bx) {
            double blk[ORC_NMAX * ORC_NMAX];
            double gap;
            const int b = by * nbx + bx;
            fsr_block_core(P, delta, out, smp, msk, psum, pcnt, H, W, by, bx, blk, 0, 0, 0, 0, 0, 0,
                           &gap, 0, follow ? follow + (size_t)b * P->iterations : NULL, bound,
                           rep ? rep + b : NULL);
            if (min_gap) min_gap[b] = gap;
            for (int m = 0; m < B; ++m)
                for (int n = 0; n < B; ++n) {
                    int y = B * by + m, x = B * bx + n;
                    if (inside(y, x, H, W)) out[(size_t)y * W + x] = blk[m * B + n];
                }
        }
}

/* The support (weights and values) of block (by, bx) with concealed weighting delta and
 * concealed values conc (H x W), for the tests. */
void orc_fsr_support(const orc_fsr_params *P, double delta, const double *conc, const uint8_t *smp,
                     const uint8_t *msk, const uint16_t *psum, const uint8_t *pcnt, int H, int W,
                     int by, int bx, double *w_out, double *f_out)
{
    fsr_support(P, delta, conc, smp, msk, psum, pcnt, H, W, by, bx, w_out, f_out);
}

/* 8-bit reconstruction: measured pixels keep their sample, all others are 255*x rounded half to
 * even and clamped to [0, 255]. */
void orc_quantize(const double *x, const uint8_t *smp, const uint8_t *msk, int H, int W,
                  uint8_t *out)
{
    for (size_t i = 0; i < (size_t)H * W; ++i) {
        if (msk[i]) { out[i] = smp[i]; continue; }
        double v = nearbyint(255.0 * x[i]);   /* default rounding mode: half to even */
        out[i] = (uint8_t)(v < 0.0 ? 0.0 : (v > 255.0 ? 255.0 : v));
    }
}
