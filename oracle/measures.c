/*
 * Oracle: plain, slow, obviously correct CPU implementation of the analyser's
 * per-pair measures.  TEST INFRASTRUCTURE ONLY: the product path (the CUDA
 * library) never links, loads or calls this file; only the tests, the smoke
 * check and the benchmark's CPU baseline do.
 *
 * Everything here is integer arithmetic, written as direct loops over the
 * definitions, with no blocking, fusion or reordering:
 *
 *   orc_downsample   pyramid level l -> l+1, (a+b+c+d+2)>>2 over 2x2 blocks,
 *                    dims floor(w/2) x floor(h/2)               (motion field, Sec. III.A)
 *   orc_sad          sum of |I - J(shifted)| over one block, J read with
 *                    clamp-to-edge addressing
 *   orc_block_search hierarchical block matching: exhaustive window at the
 *                    coarsest level, +-r refinement around twice the parent
 *                    vector at every finer level; argmin on the key
 *                    (SAD + lambda*|v|_1, |v|_1, vy, vx)         (Sec. III.A, AMM)
 *   orc_isqrt        floor(sqrt(n)) by bisection on integers
 *   orc_amm_sum      sum over blocks of floor(sqrt(dx^2+dy^2) * 2^16)    (AMM, Sec. III.A)
 *   orc_warp_sums    warp J by the block-constant field and accumulate
 *                    sum i, sum j, sum i^2, sum j^2, sum i*j, sum |i-j|  (SWR via NCC, Sec. III.A)
 *
 * The floating-point finalisation (NCC, SWR, AMM, ACT) and every decision live
 * in oracle/analyser.py.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }
static int absi(int v) { return v < 0 ? -v : v; }

/* Pyramid: one level down.  src is w x h with row pitch `pitch` bytes; dst is
 * packed (w/2) x (h/2). */
void orc_downsample(const uint8_t *src, int w, int h, long pitch, uint8_t *dst) {
    int w2 = w / 2, h2 = h / 2;
    for (int y = 0; y < h2; y++) {
        for (int x = 0; x < w2; x++) {
            int a = src[(long)(2 * y) * pitch + 2 * x];
            int b = src[(long)(2 * y) * pitch + 2 * x + 1];
            int c = src[(long)(2 * y + 1) * pitch + 2 * x];
            int d = src[(long)(2 * y + 1) * pitch + 2 * x + 1];
            dst[(long)y * w2 + x] = (uint8_t)((a + b + c + d + 2) >> 2);
        }
    }
}

/* SAD of the s x s block of I at (x0, y0) against J displaced by (vx, vy).
 * Both images are packed w x h; J is read clamp-to-edge. */
uint32_t orc_sad(const uint8_t *I, const uint8_t *J, int w, int h, int x0, int y0, int s, int vx, int vy) {
    uint32_t sad = 0;
    for (int y = 0; y < s; y++) {
        for (int x = 0; x < s; x++) {
            int i = I[(long)(y0 + y) * w + (x0 + x)];
            int jx = clampi(x0 + x + vx, 0, w - 1);
            int jy = clampi(y0 + y + vy, 0, h - 1);
            int j = J[(long)jy * w + jx];
            sad += (uint32_t)absi(i - j);
        }
    }
    return sad;
}

/* Candidate order: smaller cost = SAD + lambda*(|vx|+|vy|) first, then smaller
 * |vx|+|vy|, then smaller vy, then smaller vx (v in pixels of the level).
 * Returns nonzero when (s1,vx1,vy1) comes before (s0,vx0,vy0). */
static int better(uint32_t s1, int vx1, int vy1, uint32_t s0, int vx0, int vy0, int lambda) {
    int n1 = absi(vx1) + absi(vy1), n0 = absi(vx0) + absi(vy0);
    uint32_t c1 = s1 + (uint32_t)(lambda * n1), c0 = s0 + (uint32_t)(lambda * n0);
    if (c1 != c0) return c1 < c0;
    if (n1 != n0) return n1 < n0;
    if (vy1 != vy0) return vy1 < vy0;
    return vx1 < vx0;
}

/* Hierarchical block search.
 *   pyrI[l], pyrJ[l]  packed images of level l (l = 0 is full resolution)
 *   ws[l], hs[l]      their dims
 *   levels, block     pyramid depth L and level-0 block side B0 (B0 % 2^(L-1) == 0)
 *   R, r              coarse radius and refinement radius
 *   lambda            motion cost per pixel of |vx|+|vy| added to the SAD
 * Outputs, for the nby x nbx grid of level-0 blocks (nbx = ws[0]/B0,
 * nby = hs[0]/B0), row-major: vec[2*b] = vx, vec[2*b+1] = vy (level-0 px) and
 * sad0[b] = the SAD of the chosen level-0 vector. */
void orc_block_search(const uint8_t *const *pyrI, const uint8_t *const *pyrJ, const int *ws, const int *hs,
                      int levels, int block, int R, int r, int lambda, int16_t *vec, uint32_t *sad0) {
    int nbx = ws[0] / block, nby = hs[0] / block;
    for (int by = 0; by < nby; by++) {
        for (int bx = 0; bx < nbx; bx++) {
            int l = levels - 1;
            int s = block >> l;
            int bvx = 0, bvy = 0;
            uint32_t bsad = 0;
            int first = 1;
            for (int vy = -R; vy <= R; vy++) {
                for (int vx = -R; vx <= R; vx++) {
                    uint32_t sad = orc_sad(pyrI[l], pyrJ[l], ws[l], hs[l], bx * s, by * s, s, vx, vy);
                    if (first || better(sad, vx, vy, bsad, bvx, bvy, lambda)) {
                        bsad = sad; bvx = vx; bvy = vy; first = 0;
                    }
                }
            }
            for (l = levels - 2; l >= 0; l--) {
                s = block >> l;
                int cx = 2 * bvx, cy = 2 * bvy;
                first = 1;
                for (int dy = -r; dy <= r; dy++) {
                    for (int dx = -r; dx <= r; dx++) {
                        int vx = cx + dx, vy = cy + dy;
                        uint32_t sad = orc_sad(pyrI[l], pyrJ[l], ws[l], hs[l], bx * s, by * s, s, vx, vy);
                        if (first || better(sad, vx, vy, bsad, bvx, bvy, lambda)) {
                            bsad = sad; bvx = vx; bvy = vy; first = 0;
                        }
                    }
                }
            }
            long b = (long)by * nbx + bx;
            vec[2 * b] = (int16_t)bvx;
            vec[2 * b + 1] = (int16_t)bvy;
            if (sad0) sad0[b] = bsad;
        }
    }
}

/* floor(sqrt(n)) for n < 2^62, by bisection on the answer. */
uint64_t orc_isqrt(uint64_t n) {
    uint64_t lo = 0, hi = 1ull << 31;
    while (lo < hi) {           /* invariant: lo^2 <= n < (hi+1)^2 */
        uint64_t mid = (lo + hi + 1) / 2;
        if (mid * mid <= n) lo = mid; else hi = mid - 1;
    }
    return lo;
}

/* S_amm = sum over the nb blocks of floor(sqrt(vx^2 + vy^2) * 65536)
 *       = sum of isqrt((vx^2 + vy^2) * 2^32). */
int64_t orc_amm_sum(const int16_t *vec, long nb) {
    int64_t s = 0;
    for (long b = 0; b < nb; b++) {
        int64_t vx = vec[2 * b], vy = vec[2 * b + 1];
        uint64_t k = (uint64_t)(vx * vx + vy * vy);
        s += (int64_t)orc_isqrt(k << 32);
    }
    return s;
}

/* Motion-compensated sums over every pixel (x, y) of I (w x h, packed):
 * the block is (min(x/B0, nbx-1), min(y/B0, nby-1)), its vector v, and
 * j = J(clamp(x+vx), clamp(y+vy)).
 * sums[0..5] = sum i, sum j, sum i*i, sum j*j, sum i*j, sum |i-j|. */
void orc_warp_sums(const uint8_t *I, const uint8_t *J, int w, int h, const int16_t *vec, int nbx, int nby,
                   int block, int64_t *sums) {
    int64_t si = 0, sj = 0, sii = 0, sjj = 0, sij = 0, sad = 0;
    for (int y = 0; y < h; y++) {
        for (int x = 0; x < w; x++) {
            int bx = x / block; if (bx > nbx - 1) bx = nbx - 1;
            int by = y / block; if (by > nby - 1) by = nby - 1;
            long b = (long)by * nbx + bx;
            int vx = vec[2 * b], vy = vec[2 * b + 1];
            int64_t i = I[(long)y * w + x];
            int64_t j = J[(long)clampi(y + vy, 0, h - 1) * w + clampi(x + vx, 0, w - 1)];
            si += i; sj += j; sii += i * i; sjj += j * j; sij += i * j;
            sad += i > j ? i - j : j - i;
        }
    }
    sums[0] = si; sums[1] = sj; sums[2] = sii; sums[3] = sjj; sums[4] = sij; sums[5] = sad;
}

/* One whole pair: build both pyramids, search, AMM sum and warped sums.
 *   I0, J0  packed w x h level-0 images (frames or already-extracted fields)
 * rec[0..8] = sum i, sum j, sum i^2, sum j^2, sum i*j, sum |i-j|, S_amm, n = w*h, nb.
 * vec (optional, nby*nbx*2 int16) receives the level-0 field.
 * Returns 0, or -1 when an allocation fails or the sizes are unusable. */
int orc_pair_record(const uint8_t *I0, const uint8_t *J0, int w, int h, int levels, int block, int R, int r,
                    int lambda, int64_t *rec, int16_t *vec) {
    if (levels < 1 || levels > 8 || block <= 0 || (block % (1 << (levels - 1))) != 0) return -1;
    int nbx = w / block, nby = h / block;
    if (nbx < 1 || nby < 1) return -1;
    const uint8_t *pI[8], *pJ[8];
    uint8_t *own[16] = {0};
    int ws[8], hs[8];
    pI[0] = I0; pJ[0] = J0; ws[0] = w; hs[0] = h;
    int nown = 0, rc = 0;
    for (int l = 1; l < levels; l++) {
        ws[l] = ws[l - 1] / 2; hs[l] = hs[l - 1] / 2;
        uint8_t *a = (uint8_t *)malloc((size_t)ws[l] * hs[l] + 1);
        uint8_t *b = (uint8_t *)malloc((size_t)ws[l] * hs[l] + 1);
        own[nown++] = a; own[nown++] = b;
        if (!a || !b) { rc = -1; goto done; }
        orc_downsample(pI[l - 1], ws[l - 1], hs[l - 1], ws[l - 1], a);
        orc_downsample(pJ[l - 1], ws[l - 1], hs[l - 1], ws[l - 1], b);
        pI[l] = a; pJ[l] = b;
    }
    {
        long nb = (long)nbx * nby;
        int16_t *v = vec ? vec : (int16_t *)malloc(sizeof(int16_t) * 2 * (size_t)nb);
        if (!v) { rc = -1; goto done; }
        orc_block_search(pI, pJ, ws, hs, levels, block, R, r, lambda, v, NULL);
        int64_t sums[6];
        orc_warp_sums(I0, J0, w, h, v, nbx, nby, block, sums);
        for (int k = 0; k < 6; k++) rec[k] = sums[k];
        rec[6] = orc_amm_sum(v, nb);
        rec[7] = (int64_t)w * h;
        rec[8] = nb;
        if (!vec) free(v);
    }
done:
    for (int k = 0; k < nown; k++) free(own[k]);
    return rc;
}
