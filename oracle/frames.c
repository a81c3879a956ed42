/*
 * frames.c -- the plain, slow CPU oracle of the image front end of one
 * emulsion view: pixel filtering and 3D grain recognition.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header,
 * table or helper with the CUDA implementation, and neither imports the other.
 *
 * A view is a stack of D frames of W x H 8-bit pixels (1280 x 1024 x 40 in the
 * paper, Section 2), stored frame after frame, row after row, x fastest; rows
 * are row_pitch bytes apart.  Grains are dark in the raw image.
 *
 * Filtering (Section 2, Fig. 2b).  The pixels of the camera differ in gain, so
 * every pixel (x, y) carries its own gain g(x, y) (8 bits, 128 = 1.0) and
 * threshold t(x, y); the image is inverted.  The filtered pulse height is
 *     f = max(0, min(255, floor(((255 - raw) * g + 64) / 128)) - t).
 * (The paper names the three operations but not their form: this is the
 * plain reading, in exact integer arithmetic.)
 *
 * 3D grain recognition (Section 2, Fig. 2c).  A voxel p whose pulse height
 * exceeds the threshold T defines a grain when no voxel among its 3 x 3 x 3
 * neighbours beats it.  Voxels outside the stack do not exist.  Between equal
 * pulse heights the voxel that comes first in raster order (z, then y, then
 * x) wins, so p needs f(q) < f(p) for every neighbour q before it and
 * f(q) <= f(p) for every neighbour after it.  The grain's position is the
 * centre of mass of the neighbourhood weighted by pulse height.  Voxel index i
 * along axis k lies at i * num[k] / den[k] coordinate units; with
 * S = sum f(q) and S_k = sum f(q) * q_k over the neighbourhood, the coordinate
 * is S_k * num[k] / (S * den[k]) rounded half up:
 *     floor((2 * S_k * num[k] + S * den[k]) / (2 * S * den[k])).
 */
#include <stdint.h>
#include <stdlib.h>

enum { FR_OK = 0, FR_ERR_INVALID_ARG = -1 };

/* Filtered pulse height of one raw pixel value (the formula above). */
static int filter_px(int raw, int g, int t)
{
    int v = ((255 - raw) * g + 64) / 128;
    if (v > 255) v = 255;
    v -= t;
    return v > 0 ? v : 0;
}

/* out[(z * H + y) * W + x] = filtered value of raw[(z * H + y) * row_pitch + x]. */
int or_frames_filter(const uint8_t *raw, int64_t row_pitch, int32_t W, int32_t H, int32_t D,
                     const uint8_t *gain, const uint8_t *thr, uint8_t *out)
{
    if (!raw || !gain || !thr || !out || W <= 0 || H <= 0 || D <= 0 || row_pitch < W)
        return FR_ERR_INVALID_ARG;
    for (int64_t z = 0; z < D; ++z)
        for (int64_t y = 0; y < H; ++y)
            for (int64_t x = 0; x < W; ++x) {
                int r = raw[(z * H + y) * row_pitch + x];
                out[(z * H + y) * W + x] = (uint8_t)filter_px(r, gain[y * W + x], thr[y * W + x]);
            }
    return FR_OK;
}

/* Rounded-half-up coordinate of a centroid (see the header comment). */
static int32_t centroid_coord(int64_t sk, int64_t s, int64_t num, int64_t den)
{
    int64_t a = 2 * sk * num + s * den, b = 2 * s * den;
    int64_t q = a / b;
    if (a % b != 0 && (a < 0) != (b < 0)) --q;   /* floor; a, b > 0 here anyway */
    return (int32_t)q;
}

/* Grains of one filtered stack f (W x H x D, x fastest, no row padding), in
 * raster order of the voxel that defines them.  Writes up to cap grains:
 * xyz[3 i .. 3 i + 2], pulse[i] = S (sum of the neighbourhood's pulse
 * heights) and voxel[i] = (z * H + y) * W + x of the defining voxel.
 * Returns the number of grains (which may exceed cap), or a negative status. */
int64_t or_frames_grains(const uint8_t *f, int32_t W, int32_t H, int32_t D, int32_t T,
                         const int32_t *num, const int32_t *den, int32_t *xyz, int32_t *pulse,
                         int64_t *voxel, int64_t cap)
{
    if (!f || !num || !den || W <= 0 || H <= 0 || D <= 0 || T < 0 || cap < 0)
        return FR_ERR_INVALID_ARG;
    for (int k = 0; k < 3; ++k)
        if (num[k] <= 0 || den[k] <= 0) return FR_ERR_INVALID_ARG;
    int64_t n = 0;
    for (int64_t z = 0; z < D; ++z)
        for (int64_t y = 0; y < H; ++y)
            for (int64_t x = 0; x < W; ++x) {
                const int fp = f[(z * H + y) * W + x];
                if (fp <= T) continue;
                int is_max = 1;
                int64_t s = 0, sx = 0, sy = 0, sz = 0;
                for (int dz = -1; dz <= 1 && is_max; ++dz)
                    for (int dy = -1; dy <= 1 && is_max; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            const int64_t qx = x + dx, qy = y + dy, qz = z + dz;
                            if (qx < 0 || qx >= W || qy < 0 || qy >= H || qz < 0 || qz >= D) continue;
                            const int fq = f[(qz * H + qy) * W + qx];
                            /* q before p in raster order: the first nonzero of (dz, dy, dx) is negative */
                            const int before = dz < 0 || (dz == 0 && (dy < 0 || (dy == 0 && dx < 0)));
                            if (before ? fq >= fp : fq > fp) {
                                is_max = 0;
                                break;
                            }
                            s += fq;
                            sx += (int64_t)fq * qx;
                            sy += (int64_t)fq * qy;
                            sz += (int64_t)fq * qz;
                        }
                if (!is_max) continue;
                if (n < cap) {
                    if (xyz) {
                        xyz[3 * n + 0] = centroid_coord(sx, s, num[0], den[0]);
                        xyz[3 * n + 1] = centroid_coord(sy, s, num[1], den[1]);
                        xyz[3 * n + 2] = centroid_coord(sz, s, num[2], den[2]);
                    }
                    if (pulse) pulse[n] = (int32_t)s;
                    if (voxel) voxel[n] = (z * H + y) * W + x;
                }
                ++n;
            }
    return n;
}
