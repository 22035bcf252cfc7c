/*
 * mmr oracle: plain, slow, single-threaded C reference of the displace + render
 * hot path (Mimir benchmark, Sec. 4.1: a point cloud moved by Brownian motion
 * each timestep and drawn as same-size, same-colour markers).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this file; only the tests, the smoke check and the bench's CPU
 * baseline leg load it.  It shares no code, header or constant table with the
 * CUDA path.
 *
 * Build flags (oracle/build.py): -O2 -ffp-contract=off, no -ffast-math, SSE
 * math on x86-64, so every float operation below is one IEEE-754 binary32
 * operation rounded to nearest even, in the order written.
 *
 * Readings of the paper used here (the paper gives no formulas for them):
 *  - Displacement (Sec. 4.1 "Brownian motion"): per point i, step s, axis k,
 *    r = Philox4x32-10(ctr = (i, s, cloud, 0), key = (seed_lo, seed_hi))[k],
 *    u = (r >> 8) * 2^-24, t = 2u - 1, d = a t, p = clamp(p + d, 0, 1).
 *  - Camera: right-handed look-at view times OpenGL-style perspective, built
 *    in FP64 and rounded once to FP32 (row-major 4x4).
 *  - Projection: c = M [p, 1] with each row summed as ((m0 x + m1 y) + m2 z) + m3;
 *    kept iff znear < c.w < zfar; ndc = c.xy / c.w; sx = (ndc.x + 1)(W/2),
 *    sy = (1 - ndc.y)(H/2); inside iff 0 <= sx < W and 0 <= sy < H; pixel
 *    floor(sy) W + floor(sx) (row 0 at the top).
 *  - Splat (1-px markers, Sec. 4.1): key = bits(c.w) << 32 | id, per-pixel
 *    minimum; equal depths resolve to the smaller id.
 *  - Resolve (default colour when no colour source is bound, Sec. 3.2.2):
 *    empty pixel -> background, else colour[id] or the default colour.
 *
 * Parity pins (tests/test_oracle_pins.py): Philox against the published
 * known-answer vectors of Philox4x32-10; conversions exhaustively against
 * numpy / torch; camera and projection against closed forms and the FP64
 * twin; splat against a brute-force per-pixel search and against a shuffled
 * point order; displacement against its invariants and the FP64 twin's
 * rounding-error bound.
 */
#include <stdint.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As   */
/* Easy as 1, 2, 3", SC'11, Sec. 4.2): a 4-word counter is put through ten   */
/* rounds; each round multiplies words 0 and 2 by fixed 32-bit constants,    */
/* keeps the 64-bit products' halves and mixes the high halves with the      */
/* other two words and the round key; the 2-word key is advanced by the      */
/* Weyl constants (golden ratio, sqrt(3)-1) between rounds.                  */
/* ------------------------------------------------------------------------ */
static const uint32_t PHILOX_MUL_A = 0xD2511F53u;
static const uint32_t PHILOX_MUL_B = 0xCD9E8D57u;
static const uint32_t PHILOX_WEYL_A = 0x9E3779B9u;
static const uint32_t PHILOX_WEYL_B = 0xBB67AE85u;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_WEYL_A;
            k1 += PHILOX_WEYL_B;
        }
        uint64_t prod_a = (uint64_t)PHILOX_MUL_A * (uint64_t)x0;
        uint64_t prod_b = (uint64_t)PHILOX_MUL_B * (uint64_t)x2;
        uint32_t hi_a = (uint32_t)(prod_a >> 32), lo_a = (uint32_t)prod_a;
        uint32_t hi_b = (uint32_t)(prod_b >> 32), lo_b = (uint32_t)prod_b;
        uint32_t y0 = hi_b ^ x1 ^ k0;
        uint32_t y1 = lo_b;
        uint32_t y2 = hi_a ^ x3 ^ k1;
        uint32_t y3 = lo_a;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Philox4x32-10 of n counters with their keys (ctr: 4n words, key: 2n). */
void orc_philox4x32_10_many(const uint32_t *ctr, const uint32_t *key, uint32_t *out, uint64_t n)
{
    for (uint64_t i = 0; i < n; ++i)
        orc_philox4x32_10(ctr + 4 * i, key + 2 * i, out + 4 * i);
}

/* The three 32-bit draws that move point `i` at step `s` (Sec. 4.1). */
static void draws_for_point(uint64_t seed, uint32_t cloud, uint32_t i, uint32_t s, uint32_t r[4])
{
    uint32_t ctr[4] = { i, s, cloud, 0u };
    uint32_t key[2] = { (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) };
    orc_philox4x32_10(ctr, key, r);
}

/* ------------------------------------------------------------------------ */
/* Displacement, FP32 (Sec. 4.1).  One axis: top 24 bits of the draw give a  */
/* uniform u in [0, 1 - 2^-24]; t = 2u - 1; d = a t; p = clamp(p + d, 0, 1).  */
/* ------------------------------------------------------------------------ */
static float uniform24_f32(uint32_t r)
{
    return (float)(r >> 8) * 0x1p-24f;   /* exact: a 24-bit integer times 2^-24 */
}

/* The clamp to [0, 1] takes IEEE 754 maxNum / minNum (C's fmaxf / fminf):
 * +inf -> 1, -inf -> 0, and a NaN coordinate, which only a caller's own NaN
 * input can produce, -> 0, so every coordinate stays in the unit box.       */
static float move_axis_f32(float p, uint32_t r, float a)
{
    float u = uniform24_f32(r);
    float t = 2.0f * u;
    t = t + (-1.0f);
    float d = a * t;
    float q = p + d;
    return fminf(fmaxf(q, 0.0f), 1.0f);
}

void orc_displace_f32(float *pos, uint64_t n, uint64_t seed, uint32_t cloud, uint32_t step, float a)
{
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t r[4];
        draws_for_point(seed, cloud, (uint32_t)i, step, r);
        for (int k = 0; k < 3; ++k)
            pos[3 * i + k] = move_axis_f32(pos[3 * i + k], r[k], a);
    }
}

/* Displace only the points listed in `ids` (positions packed in the same
 * order as `ids`); used to follow sampled points through many steps. */
void orc_displace_ids_f32(float *pos, const uint32_t *ids, uint64_t m, uint64_t seed,
                          uint32_t cloud, uint32_t step, float a)
{
    for (uint64_t j = 0; j < m; ++j) {
        uint32_t r[4];
        draws_for_point(seed, cloud, ids[j], step, r);
        for (int k = 0; k < 3; ++k)
            pos[3 * j + k] = move_axis_f32(pos[3 * j + k], r[k], a);
    }
}

/* The same iteration in FP64: identical draws, every operation in double. */
void orc_displace_f64(double *pos, uint64_t n, uint64_t seed, uint32_t cloud, uint32_t step, double a)
{
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t r[4];
        draws_for_point(seed, cloud, (uint32_t)i, step, r);
        for (int k = 0; k < 3; ++k) {
            double u = (double)(r[k] >> 8) * 0x1p-24;
            double t = 2.0 * u - 1.0;
            double q = pos[3 * i + k] + a * t;
            if (q < 0.0) q = 0.0;
            if (q > 1.0) q = 1.0;
            pos[3 * i + k] = q;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Storage conversions, written from the IEEE-754 binary16 and bfloat16      */
/* formats: binary16 has 1 sign, 5 exponent (bias 15), 10 fraction bits;     */
/* bfloat16 is the top 16 bits of binary32.  Narrowing rounds to nearest,    */
/* ties to even.                                                             */
/* ------------------------------------------------------------------------ */
static uint32_t f32_bits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static float bits_f32(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }

uint16_t orc_f32_to_f16(float f)
{
    uint32_t x = f32_bits(f);
    uint32_t sign = (x >> 16) & 0x8000u;
    uint32_t mag = x & 0x7fffffffu;
    if (mag > 0x7f800000u)                 /* NaN: quiet NaN, keep top payload bits */
        return (uint16_t)(sign | 0x7e00u | ((mag >> 13) & 0x3ffu));
    if (mag >= 0x477ff000u)                /* >= 65520 rounds past 65504: infinity */
        return (uint16_t)(sign | 0x7c00u);
    if (mag >= 0x38800000u) {              /* >= 2^-14: normal binary16 */
        uint32_t e = (mag >> 23) - 127u + 15u;
        uint32_t frac = mag & 0x7fffffu;
        uint32_t h = (e << 10) | (frac >> 13);
        uint32_t rest = frac & 0x1fffu;
        if (rest > 0x1000u || (rest == 0x1000u && (h & 1u)))
            h += 1u;                       /* a carry into the exponent is correct */
        return (uint16_t)(sign | h);
    }
    if (mag <= 0x33000000u)                /* <= 2^-25: rounds to zero (tie -> even 0) */
        return (uint16_t)sign;
    /* Subnormal result: value = m * 2^(e-150); in units of 2^-24 that is
     * m * 2^(e-126), a right shift of 126 - e bits (14..24). */
    uint32_t e = mag >> 23;
    uint32_t m = (mag & 0x7fffffu) | 0x800000u;
    uint32_t shift = 126u - e;
    uint32_t h = m >> shift;
    uint32_t rest = m & ((1u << shift) - 1u);
    uint32_t half = 1u << (shift - 1u);
    if (rest > half || (rest == half && (h & 1u)))
        h += 1u;
    return (uint16_t)(sign | h);
}

float orc_f16_to_f32(uint16_t h)
{
    uint32_t sign = ((uint32_t)h & 0x8000u) << 16;
    uint32_t e = ((uint32_t)h >> 10) & 0x1fu;
    uint32_t frac = (uint32_t)h & 0x3ffu;
    if (e == 0x1fu)
        return bits_f32(sign | 0x7f800000u | (frac << 13));
    if (e == 0u) {
        float v = (float)frac * 0x1p-24f;  /* exact: frac < 2^10 */
        return sign ? -v : v;
    }
    return bits_f32(sign | ((e - 15u + 127u) << 23) | (frac << 13));
}

uint16_t orc_f32_to_bf16(float f)
{
    uint32_t x = f32_bits(f);
    if ((x & 0x7fffffffu) > 0x7f800000u)   /* NaN: quiet it */
        return (uint16_t)((x >> 16) | 0x0040u);
    uint32_t keep = x >> 16;
    uint32_t rest = x & 0xffffu;
    if (rest > 0x8000u || (rest == 0x8000u && (keep & 1u)))
        keep += 1u;                        /* carries reach the exponent / infinity */
    return (uint16_t)keep;
}

float orc_bf16_to_f32(uint16_t b) { return bits_f32((uint32_t)b << 16); }

void orc_f32_to_f16_array(const float *src, uint16_t *dst, uint64_t n)
{ for (uint64_t i = 0; i < n; ++i) dst[i] = orc_f32_to_f16(src[i]); }
void orc_f16_to_f32_array(const uint16_t *src, float *dst, uint64_t n)
{ for (uint64_t i = 0; i < n; ++i) dst[i] = orc_f16_to_f32(src[i]); }
void orc_f32_to_bf16_array(const float *src, uint16_t *dst, uint64_t n)
{ for (uint64_t i = 0; i < n; ++i) dst[i] = orc_f32_to_bf16(src[i]); }
void orc_bf16_to_f32_array(const uint16_t *src, float *dst, uint64_t n)
{ for (uint64_t i = 0; i < n; ++i) dst[i] = orc_bf16_to_f32(src[i]); }

/* Displacement with 16-bit storage: widen exactly, move in FP32, narrow RNE.
 * kind 1 = binary16, kind 2 = bfloat16. */
void orc_displace_h16(uint16_t *pos, int kind, uint64_t n, uint64_t seed, uint32_t cloud,
                      uint32_t step, float a)
{
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t r[4];
        draws_for_point(seed, cloud, (uint32_t)i, step, r);
        for (int k = 0; k < 3; ++k) {
            float p = kind == 1 ? orc_f16_to_f32(pos[3 * i + k]) : orc_bf16_to_f32(pos[3 * i + k]);
            float q = move_axis_f32(p, r[k], a);
            pos[3 * i + k] = kind == 1 ? orc_f32_to_f16(q) : orc_f32_to_bf16(q);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Camera: look-at view matrix V and perspective P, both FP64, M = P V.      */
/*   f = normalize(target - eye), s = normalize(f x up), u = s x f           */
/*   V rows: (s, -s.eye), (u, -u.eye), (-f, f.eye), (0,0,0,1)                */
/*   P: diag(g/aspect, g), g = 1/tan(fovy/2); z row ((zf+zn)/(zn-zf),        */
/*      2 zf zn/(zn-zf)); w row (0, 0, -1, 0), so clip w = f.(p - eye).      */
/* ------------------------------------------------------------------------ */
static void normalize3(double v[3])
{
    double len = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] /= len; v[1] /= len; v[2] /= len;
}

static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

void orc_camera_f64(const double eye[3], const double target[3], const double up[3],
                    double fovy_deg, double aspect, double znear, double zfar, double M[16])
{
    double f[3] = { target[0] - eye[0], target[1] - eye[1], target[2] - eye[2] };
    normalize3(f);
    double s[3];
    cross3(f, up, s);
    normalize3(s);
    double u[3];
    cross3(s, f, u);
    double V[16] = {
        s[0], s[1], s[2], -dot3(s, eye),
        u[0], u[1], u[2], -dot3(u, eye),
        -f[0], -f[1], -f[2], dot3(f, eye),
        0.0, 0.0, 0.0, 1.0,
    };
    const double pi = 3.14159265358979323846;
    double g = 1.0 / tan(0.5 * fovy_deg * (pi / 180.0));
    double P[16] = {
        g / aspect, 0.0, 0.0, 0.0,
        0.0, g, 0.0, 0.0,
        0.0, 0.0, (zfar + znear) / (znear - zfar), 2.0 * zfar * znear / (znear - zfar),
        0.0, 0.0, -1.0, 0.0,
    };
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            double acc = 0.0;
            for (int k = 0; k < 4; ++k)
                acc += P[4 * r + k] * V[4 * k + c];
            M[4 * r + c] = acc;
        }
}

void orc_camera_f32(const double eye[3], const double target[3], const double up[3],
                    double fovy_deg, double aspect, double znear, double zfar, float M32[16])
{
    double M[16];
    orc_camera_f64(eye, target, up, fovy_deg, aspect, znear, zfar, M);
    for (int k = 0; k < 16; ++k)
        M32[k] = (float)M[k];              /* the one rounding FP64 -> FP32 */
}

/* ------------------------------------------------------------------------ */
/* Projection of one point, FP32 in the stated order.  Returns 1 and the     */
/* pixel index and clip w when the point lands inside the W x H frame.       */
/* ------------------------------------------------------------------------ */
int orc_project_f32(const float M[16], float x, float y, float z, int W, int H,
                    float znear, float zfar, uint32_t *px, float *w_out, float ndc[2])
{
    float cx = ((M[0] * x + M[1] * y) + M[2] * z) + M[3];
    float cy = ((M[4] * x + M[5] * y) + M[6] * z) + M[7];
    float cw = ((M[12] * x + M[13] * y) + M[14] * z) + M[15];
    if (!(cw > znear && cw < zfar))
        return 0;
    float nx = cx / cw;
    float ny = cy / cw;
    if (ndc) { ndc[0] = nx; ndc[1] = ny; }
    float sx = (nx + 1.0f) * (0.5f * (float)W);
    float sy = (1.0f - ny) * (0.5f * (float)H);
    if (!(sx >= 0.0f && sx < (float)W && sy >= 0.0f && sy < (float)H))
        return 0;
    *px = (uint32_t)(int)sy * (uint32_t)W + (uint32_t)(int)sx;
    *w_out = cw;
    return 1;
}

/* The FP64 twin used to bound the FP32 projection error. */
int orc_project_f64(const double M[16], double x, double y, double z, double znear, double zfar,
                    double ndc[2], double *w_out)
{
    double cx = M[0] * x + M[1] * y + M[2] * z + M[3];
    double cy = M[4] * x + M[5] * y + M[6] * z + M[7];
    double cw = M[12] * x + M[13] * y + M[14] * z + M[15];
    if (!(cw > znear && cw < zfar))
        return 0;
    ndc[0] = cx / cw;
    ndc[1] = cy / cw;
    *w_out = cw;
    return 1;
}

/* Batch helper for the tests: project n FP32 points; px = 0xffffffff when
 * the point is culled or off-frame. */
void orc_project_many_f32(const float M[16], const float *pos, uint64_t n, int W, int H,
                          float znear, float zfar, uint32_t *px, float *w, float *ndc)
{
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t p; float cw; float nd[2] = { 0.0f, 0.0f };
        if (orc_project_f32(M, pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], W, H, znear, zfar,
                            &p, &cw, nd)) {
            px[i] = p; w[i] = cw;
        } else {
            px[i] = 0xffffffffu; w[i] = 0.0f;
        }
        if (ndc) { ndc[2 * i] = nd[0]; ndc[2 * i + 1] = nd[1]; }
    }
}

void orc_project_many_f64(const double M[16], const double *pos, uint64_t n, double znear,
                          double zfar, double *ndc, double *w, int32_t *valid)
{
    for (uint64_t i = 0; i < n; ++i) {
        double nd[2] = { 0.0, 0.0 }, cw = 0.0;
        valid[i] = orc_project_f64(M, pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], znear, zfar, nd, &cw);
        ndc[2 * i] = nd[0]; ndc[2 * i + 1] = nd[1]; w[i] = cw;
    }
}

/* ------------------------------------------------------------------------ */
/* Splat: per-pixel minimum of key = bits(w) << 32 | (id_base + i).          */
/* keybuf must start at all-ones for an empty frame.                         */
/* ------------------------------------------------------------------------ */
void orc_splat_f32(const float *pos, uint64_t n, const float M[16], int W, int H,
                   float znear, float zfar, uint32_t id_base, uint64_t *keybuf)
{
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t px; float cw;
        if (!orc_project_f32(M, pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], W, H, znear, zfar,
                             &px, &cw, 0))
            continue;
        uint64_t key = ((uint64_t)f32_bits(cw) << 32) | (uint64_t)(uint32_t)(id_base + (uint32_t)i);
        if (key < keybuf[px])
            keybuf[px] = key;
    }
}

void orc_splat_h16(const uint16_t *pos, int kind, uint64_t n, const float M[16], int W, int H,
                   float znear, float zfar, uint32_t id_base, uint64_t *keybuf)
{
    for (uint64_t i = 0; i < n; ++i) {
        float p[3];
        for (int k = 0; k < 3; ++k)
            p[k] = kind == 1 ? orc_f16_to_f32(pos[3 * i + k]) : orc_bf16_to_f32(pos[3 * i + k]);
        uint32_t px; float cw;
        if (!orc_project_f32(M, p[0], p[1], p[2], W, H, znear, zfar, &px, &cw, 0))
            continue;
        uint64_t key = ((uint64_t)f32_bits(cw) << 32) | (uint64_t)(uint32_t)(id_base + (uint32_t)i);
        if (key < keybuf[px])
            keybuf[px] = key;
    }
}

/* Disc markers of radius r pixels (the paper's front-facing disc markers,
 * Sec. 4.1): the point's key goes to every pixel whose centre (px + 1/2,
 * py + 1/2) lies within r of the projected point (sx, sy):
 *   dx = (px + 1/2) - sx, dy = (py + 1/2) - sy, covered iff dx*dx + dy*dy <= r*r
 * in FP32, in that order.  The candidate pixels are those of the box
 * [sx - r - 1, sx + r + 1] x [sy - r - 1, sy + r + 1] clipped to the frame; the
 * exact test decides.  Depth and id as for 1-px points. */
static int screen_f32(const float M[16], float x, float y, float z, float halfW, float halfH, float znear, float zfar,
                      float *sx, float *sy, float *cw_out)
{
    float cx = ((M[0] * x + M[1] * y) + M[2] * z) + M[3];
    float cy = ((M[4] * x + M[5] * y) + M[6] * z) + M[7];
    float cw = ((M[12] * x + M[13] * y) + M[14] * z) + M[15];
    if (!(cw > znear && cw < zfar))
        return 0;
    float nx = cx / cw;
    float ny = cy / cw;
    *sx = (nx + 1.0f) * halfW;
    *sy = (1.0f - ny) * halfH;
    *cw_out = cw;
    return 1;
}

void orc_splat_disc_f32(const float *pos, uint64_t n, const float M[16], int W, int H, float znear, float zfar,
                        float radius, uint32_t id_base, uint64_t *keybuf)
{
    const float r2 = radius * radius;
    const float halfW = 0.5f * (float)W, halfH = 0.5f * (float)H;
    for (uint64_t i = 0; i < n; ++i) {
        float sx, sy, cw;
        if (!screen_f32(M, pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], halfW, halfH, znear, zfar, &sx, &sy, &cw))
            continue;
        float xa = sx - radius - 1.0f, xb = sx + radius + 1.0f;
        float ya = sy - radius - 1.0f, yb = sy + radius + 1.0f;
        if (xa < 0.0f) xa = 0.0f;
        if (ya < 0.0f) ya = 0.0f;
        if (xb > (float)(W - 1)) xb = (float)(W - 1);
        if (yb > (float)(H - 1)) yb = (float)(H - 1);
        if (!(xa <= xb && ya <= yb))
            continue;
        uint64_t key = ((uint64_t)f32_bits(cw) << 32) | (uint64_t)(uint32_t)(id_base + (uint32_t)i);
        for (int py = (int)ya; py <= (int)yb; ++py) {
            float dy = ((float)py + 0.5f) - sy;
            for (int px = (int)xa; px <= (int)xb; ++px) {
                float dx = ((float)px + 0.5f) - sx;
                float d2 = dx * dx + dy * dy;
                if (d2 <= r2) {
                    uint64_t *k = &keybuf[(uint64_t)py * (uint64_t)W + (uint64_t)px];
                    if (key < *k)
                        *k = key;
                }
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Second workload: gravitational all-pairs N-body (the paper's N-body       */
/* sample, Sec. 4.2.3), written from the physics.  Softened Newtonian        */
/* gravity; for body i the terms, j = 0 .. n-1,                              */
/*   d = p_j - p_i,  r2 = ((dx dx + dy dy) + dz dz) + eps2,                  */
/*   inv = 1 / sqrt(r2),  t_j = d (m_j ((inv inv) inv))   (zero for j = i),  */
/* summed in order of j, acc = (..((t_0 + t_1) + t_2) ..) + t_{n-1}.  Then   */
/* a = G acc, v' = v + a dt, p' = p + v' dt (semi-implicit Euler).  FP32,    */
/* every operation rounded once, in that order; positions are read from pin */
/* and written to pout (two buffers, as the paper's ping-pong).              */
/* ------------------------------------------------------------------------ */

/* One term t_j of body i's sum (shared by the two summation orders below). */
static void nbody_term(const float *pin, const float *mass, uint64_t j, float px, float py, float pz, float eps2,
                       float t[3])
{
    float dx = pin[3 * j] - px;
    float dy = pin[3 * j + 1] - py;
    float dz = pin[3 * j + 2] - pz;
    float r2 = ((dx * dx + dy * dy) + dz * dz) + eps2;
    float inv = 1.0f / sqrtf(r2);
    float s = mass[j] * ((inv * inv) * inv);
    t[0] = dx * s;
    t[1] = dy * s;
    t[2] = dz * s;
}

/* The update of body i from its summed acceleration (ax, ay, az). */
static void nbody_update(const float *pin, float *pout, float *vel, uint64_t i, float ax, float ay, float az,
                         float G, float dt)
{
    float vx = vel[3 * i] + (G * ax) * dt;
    float vy = vel[3 * i + 1] + (G * ay) * dt;
    float vz = vel[3 * i + 2] + (G * az) * dt;
    vel[3 * i] = vx;
    vel[3 * i + 1] = vy;
    vel[3 * i + 2] = vz;
    pout[3 * i] = pin[3 * i] + vx * dt;
    pout[3 * i + 1] = pin[3 * i + 1] + vy * dt;
    pout[3 * i + 2] = pin[3 * i + 2] + vz * dt;
}

/* The definition: the plain sequential sum over j. */
void orc_nbody_step_f32(const float *pin, float *pout, float *vel, const float *mass, uint64_t n, float G,
                        float eps2, float dt)
{
    for (uint64_t i = 0; i < n; ++i) {
        const float px = pin[3 * i], py = pin[3 * i + 1], pz = pin[3 * i + 2];
        float ax = 0.0f, ay = 0.0f, az = 0.0f, t[3];
        for (uint64_t j = 0; j < n; ++j) {
            nbody_term(pin, mass, j, px, py, pz, eps2, t);
            ax = ax + t[0];
            ay = ay + t[1];
            az = az + t[2];
        }
        nbody_update(pin, pout, vel, i, ax, ay, az, G, dt);
    }
}

/* The same terms summed in another fixed order, the one a GPU kernel uses:  */
/* chunks of `chunk` consecutive j, each chunk in order of j from zero, then */
/* the chunk sums in chunk order from zero.  With one chunk it is the        */
/* sequential sum above.  This is not a second definition: it replays the    */
/* kernel's rounding order so the kernel can be checked bit for bit, while   */
/* the kernel is held to the sequential sum by a summation error bound.      */
void orc_nbody_step_f32_chunked(const float *pin, float *pout, float *vel, const float *mass, uint64_t n, float G,
                                float eps2, float dt, uint64_t chunk)
{
    for (uint64_t i = 0; i < n; ++i) {
        const float px = pin[3 * i], py = pin[3 * i + 1], pz = pin[3 * i + 2];
        float ax = 0.0f, ay = 0.0f, az = 0.0f, t[3];
        for (uint64_t c0 = 0; c0 < n; c0 += chunk) {
            const uint64_t c1 = c0 + chunk < n ? c0 + chunk : n;
            float sx = 0.0f, sy = 0.0f, sz = 0.0f;
            for (uint64_t j = c0; j < c1; ++j) {
                nbody_term(pin, mass, j, px, py, pz, eps2, t);
                sx = sx + t[0];
                sy = sy + t[1];
                sz = sz + t[2];
            }
            ax = ax + sx;
            ay = ay + sy;
            az = az + sz;
        }
        nbody_update(pin, pout, vel, i, ax, ay, az, G, dt);
    }
}

/* Sum over j of |t_j| per component, in FP64 from the FP32 terms (the      */
/* magnitudes a summation error bound scales with).                          */
void orc_nbody_abs_term_sums(const float *pin, const float *mass, uint64_t n, float eps2, double *out)
{
    for (uint64_t i = 0; i < n; ++i) {
        double a[3] = { 0.0, 0.0, 0.0 };
        float t[3];
        for (uint64_t j = 0; j < n; ++j) {
            nbody_term(pin, mass, j, pin[3 * i], pin[3 * i + 1], pin[3 * i + 2], eps2, t);
            for (int k = 0; k < 3; ++k)
                a[k] += fabs((double)t[k]);
        }
        for (int k = 0; k < 3; ++k)
            out[3 * i + k] = a[k];
    }
}

/* FP64 accelerations G * sum_j m_j d / (|d|^2 + eps2)^(3/2), for the pins. */
void orc_nbody_accel_f64(const double *p, const double *mass, uint64_t n, double G, double eps2, double *acc)
{
    for (uint64_t i = 0; i < n; ++i) {
        double a[3] = { 0.0, 0.0, 0.0 };
        for (uint64_t j = 0; j < n; ++j) {
            double d[3] = { p[3 * j] - p[3 * i], p[3 * j + 1] - p[3 * i + 1], p[3 * j + 2] - p[3 * i + 2] };
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + eps2;
            double s = mass[j] / (r2 * sqrt(r2));
            for (int k = 0; k < 3; ++k)
                a[k] += d[k] * s;
        }
        for (int k = 0; k < 3; ++k)
            acc[3 * i + k] = G * a[k];
    }
}

/* Resolve: key -> RGBA8.  colors == NULL means every point takes `color`. */
void orc_resolve(const uint64_t *keybuf, uint64_t npx, const uint32_t *colors, uint32_t color,
                 uint32_t background, uint32_t *rgba)
{
    for (uint64_t p = 0; p < npx; ++p) {
        uint64_t key = keybuf[p];
        if (key == ~(uint64_t)0)
            rgba[p] = background;
        else
            rgba[p] = colors ? colors[(uint32_t)(key & 0xffffffffu)] : color;
    }
}

/* One whole frame in FP32 storage: displace (step s), clear, splat, resolve. */
void orc_frame_f32(float *pos, uint64_t n, uint64_t seed, uint32_t cloud, uint32_t step, float a,
                   const float M[16], int W, int H, float znear, float zfar, const uint32_t *colors,
                   uint32_t color, uint32_t background, uint64_t *keybuf, uint32_t *rgba)
{
    orc_displace_f32(pos, n, seed, cloud, step, a);
    uint64_t npx = (uint64_t)W * (uint64_t)H;
    for (uint64_t p = 0; p < npx; ++p)
        keybuf[p] = ~(uint64_t)0;
    orc_splat_f32(pos, n, M, W, H, znear, zfar, 0u, keybuf);
    orc_resolve(keybuf, npx, colors, color, background, rgba);
}
