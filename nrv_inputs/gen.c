/*
 * Seeded synthetic inputs: point clouds, attribute streams and network weights.
 *
 * This file generates INPUTS only.  It holds none of the rendering method's
 * arithmetic (no projection, visibility, resolve, packing or network math):
 * both the CUDA library and the CPU oracle consume what it writes.
 *
 * Every value is a pure function of (seed, stream, index), so the output does
 * not depend on the number of OpenMP threads.  Random numbers come from
 * SplitMix64 (Steele, Lea, Flood 2014): the i-th output of a SplitMix64
 * sequence whose state starts at s is mix(s + (i+1)*gamma).  A stream's state
 * is itself the stream-th output of the sequence seeded with `seed`.
 *
 * Built with -ffp-contract=off so that x86 and Arm hosts give the same floats.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GAMMA 0x9E3779B97F4A7C15ull

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t nrvi_bits(uint64_t seed, uint64_t stream, uint64_t index) {
    uint64_t key = mix64(seed + (stream + 1) * GAMMA);
    return mix64(key + (index + 1) * GAMMA);
}

/* 53-bit uniform double in [0, 1). */
double nrvi_uniform(uint64_t seed, uint64_t stream, uint64_t index) {
    return (double)(nrvi_bits(seed, stream, index) >> 11) * 0x1.0p-53;
}

/* Box-Muller standard normal from the uniforms at indices 2i and 2i+1. */
double nrvi_normal(uint64_t seed, uint64_t stream, uint64_t index) {
    double u1 = nrvi_uniform(seed, stream, 2 * index);
    double u2 = nrvi_uniform(seed, stream, 2 * index + 1);
    return sqrt(-2.0 * log(1.0 - u1)) * cos(6.283185307179586 * u2);
}

static inline uint32_t f2u(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

/* out[i*stride] = (float)(lo + (hi-lo)*U), as float bits when out is a word array. */
void nrvi_fill_uniform(uint64_t seed, uint64_t stream, int64_t n, double lo, double hi,
                       float* out, int64_t stride) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        out[i * stride] = (float)(lo + (hi - lo) * nrvi_uniform(seed, stream, (uint64_t)i));
}

void nrvi_fill_normal(uint64_t seed, uint64_t stream, int64_t n, float* out, int64_t stride) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        out[i * stride] = (float)nrvi_normal(seed, stream, (uint64_t)i);
}

/* Uniform points in the unit cube: x, y, z from streams 0, 1, 2. */
void nrvi_cube_points(uint64_t seed, int64_t n, float* xyz) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        xyz[3 * i + 0] = (float)nrvi_uniform(seed, 0, (uint64_t)i);
        xyz[3 * i + 1] = (float)nrvi_uniform(seed, 1, (uint64_t)i);
        xyz[3 * i + 2] = (float)nrvi_uniform(seed, 2, (uint64_t)i);
    }
}

/*
 * Static vector field: a jittered g^3 grid in the unit cube (x fastest), and a
 * Rankine vortex about the vertical (y) axis through x = z = 0.5 with core radius
 * R = 0.1 and circulation 2*pi*R (peak speed 1), plus N(0, sigma^2) noise per
 * velocity component.  Record words: vx, vy, vz, |v_noisy|, pressure, then zero
 * padding up to stride_words.  Pressure is the analytic Rankine pressure with
 * rho = 1 and zero pressure at infinity.
 */
void nrvi_vortex_grid(int64_t g, uint64_t seed, double sigma, float* xyz, uint32_t* attr,
                      int64_t stride_words) {
    const double R = 0.1;
    int64_t n = g * g * g;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int64_t ix = i % g, iy = (i / g) % g, iz = i / (g * g);
        double x = ((double)ix + nrvi_uniform(seed, 0, (uint64_t)i)) / (double)g;
        double y = ((double)iy + nrvi_uniform(seed, 1, (uint64_t)i)) / (double)g;
        double z = ((double)iz + nrvi_uniform(seed, 2, (uint64_t)i)) / (double)g;
        float fx = (float)x, fy = (float)y, fz = (float)z;
        xyz[3 * i + 0] = fx; xyz[3 * i + 1] = fy; xyz[3 * i + 2] = fz;
        double dx = (double)fx - 0.5, dz = (double)fz - 0.5;
        double r = sqrt(dx * dx + dz * dz);
        double vth = r <= R ? r / R : R / r;
        double vx = 0.0, vz = 0.0;
        if (r > 0.0) { vx = vth * dz / r; vz = -vth * dx / r; }
        double p = r <= R ? -0.5 * (2.0 - r * r / (R * R)) : -0.5 * R * R / (r * r);
        vx += sigma * nrvi_normal(seed, 3, (uint64_t)i);
        double vy = sigma * nrvi_normal(seed, 4, (uint64_t)i);
        vz += sigma * nrvi_normal(seed, 5, (uint64_t)i);
        double sp = sqrt(vx * vx + vy * vy + vz * vz);
        uint32_t* rec = attr + i * stride_words;
        rec[0] = f2u((float)vx); rec[1] = f2u((float)vy); rec[2] = f2u((float)vz);
        rec[3] = f2u((float)sp); rec[4] = f2u((float)p);
        for (int64_t w = 5; w < stride_words; ++w) rec[w] = 0u;
    }
}

/*
 * Vortex set for the trajectory scene.  Per vortex k (8 doubles):
 * centre ~ U[0,1)^3, unit axis uniform on the sphere, R ~ U[0.05, 0.2],
 * circulation Gamma ~ U[-1, 1] * 2*pi*R.  Streams 200 + 8k + j.
 */
void nrvi_vortex_params(uint64_t seed, int nv, double* out) {
    for (int k = 0; k < nv; ++k) {
        uint64_t s = 200 + 8 * (uint64_t)k;
        double* v = out + 8 * k;
        v[0] = nrvi_uniform(seed, s + 0, 0);
        v[1] = nrvi_uniform(seed, s + 1, 0);
        v[2] = nrvi_uniform(seed, s + 2, 0);
        double zc = 2.0 * nrvi_uniform(seed, s + 3, 0) - 1.0;
        double ph = 6.283185307179586 * nrvi_uniform(seed, s + 4, 0);
        double rs = sqrt(1.0 - zc * zc);
        v[3] = rs * cos(ph); v[4] = rs * sin(ph); v[5] = zc;
        v[6] = 0.05 + 0.15 * nrvi_uniform(seed, s + 5, 0);
        v[7] = (2.0 * nrvi_uniform(seed, s + 6, 0) - 1.0) * 6.283185307179586 * v[6];
    }
}

/* Sum of Rankine swirls about each vortex line. */
static void swirl_field(const double* vort, int nv, const double p[3], double v[3]) {
    v[0] = v[1] = v[2] = 0.0;
    for (int k = 0; k < nv; ++k) {
        const double* q = vort + 8 * k;
        double d0 = p[0] - q[0], d1 = p[1] - q[1], d2 = p[2] - q[2];
        double al = d0 * q[3] + d1 * q[4] + d2 * q[5];
        double r0 = d0 - al * q[3], r1 = d1 - al * q[4], r2 = d2 - al * q[5];
        double r = sqrt(r0 * r0 + r1 * r1 + r2 * r2);
        if (r <= 0.0) continue;
        double R = q[6], G = q[7];
        double vth = r <= R ? G / (6.283185307179586 * R) * (r / R) : G / (6.283185307179586 * r);
        /* direction = axis x r_vec / r */
        double c0 = q[4] * r2 - q[5] * r1, c1 = q[5] * r0 - q[3] * r2, c2 = q[3] * r1 - q[4] * r0;
        v[0] += vth * c0 / r; v[1] += vth * c1 / r; v[2] += vth * c2 / r;
    }
}

/*
 * Particle trajectories: np particles start U[0,1)^3 (streams 0..2), are advected
 * by classic RK4 in double through the vortex field for ns steps of dt, and the
 * position after each step is stored (particle-major: point = particle*ns + s).
 * Record words: t = (s+1)*dt (f32), |v| at the stored position (f32), particle
 * id (u32), then zero padding up to stride_words.
 */
void nrvi_trajectories(int64_t np, int64_t ns, double dt, uint64_t seed, const double* vort,
                       int nv, float* xyz, uint32_t* attr, int64_t stride_words) {
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t pi = 0; pi < np; ++pi) {
        double p[3] = {nrvi_uniform(seed, 0, (uint64_t)pi), nrvi_uniform(seed, 1, (uint64_t)pi),
                       nrvi_uniform(seed, 2, (uint64_t)pi)};
        for (int64_t s = 0; s < ns; ++s) {
            double k1[3], k2[3], k3[3], k4[3], t[3];
            swirl_field(vort, nv, p, k1);
            for (int j = 0; j < 3; ++j) t[j] = p[j] + 0.5 * dt * k1[j];
            swirl_field(vort, nv, t, k2);
            for (int j = 0; j < 3; ++j) t[j] = p[j] + 0.5 * dt * k2[j];
            swirl_field(vort, nv, t, k3);
            for (int j = 0; j < 3; ++j) t[j] = p[j] + dt * k3[j];
            swirl_field(vort, nv, t, k4);
            for (int j = 0; j < 3; ++j) p[j] += dt / 6.0 * (k1[j] + 2.0 * k2[j] + 2.0 * k3[j] + k4[j]);
            double v[3];
            swirl_field(vort, nv, p, v);
            int64_t i = pi * ns + s;
            xyz[3 * i + 0] = (float)p[0]; xyz[3 * i + 1] = (float)p[1]; xyz[3 * i + 2] = (float)p[2];
            uint32_t* rec = attr + i * stride_words;
            rec[0] = f2u((float)((double)(s + 1) * dt));
            rec[1] = f2u((float)sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
            rec[2] = (uint32_t)pi;
            for (int64_t w = 3; w < stride_words; ++w) rec[w] = 0u;
        }
    }
}

/* ---- terrain ---------------------------------------------------------- */

static inline double smooth(double t) { return t * t * (3.0 - 2.0 * t); }

static double lattice(uint64_t seed, int oct, int64_t ix, int64_t iz) {
    uint64_t idx = ((uint64_t)(ix + 1048576) << 21) ^ (uint64_t)(iz + 1048576);
    return 2.0 * nrvi_uniform(seed, 100 + (uint64_t)oct, idx) - 1.0;
}

static double value_noise(uint64_t seed, int oct, double u, double v) {
    double fu = floor(u), fv = floor(v);
    int64_t iu = (int64_t)fu, iv = (int64_t)fv;
    double a = smooth(u - fu), b = smooth(v - fv);
    double l00 = lattice(seed, oct, iu, iv), l10 = lattice(seed, oct, iu + 1, iv);
    double l01 = lattice(seed, oct, iu, iv + 1), l11 = lattice(seed, oct, iu + 1, iv + 1);
    double top = l00 + (l10 - l00) * a, bot = l01 + (l11 - l01) * a;
    return top + (bot - top) * b;
}

/* 6-octave fBm of value noise: lacunarity 2, gain 0.5, base wavelength 2.5 km, amplitude 400 m. */
double nrvi_terrain_height(uint64_t seed, double x, double z) {
    double h = 0.0, amp = 400.0, f = 1.0 / 2500.0;
    for (int o = 0; o < 6; ++o) {
        h += amp * value_noise(seed, o, x * f, z * f);
        amp *= 0.5; f *= 2.0;
    }
    return h;
}

/* Five height bands (metres) -> RGB, packed little-endian R | G<<8 | B<<16 | 255<<24. */
uint32_t nrvi_band_colour(double h) {
    static const uint8_t c[5][3] = {{40, 70, 160}, {194, 178, 128}, {80, 140, 60},
                                    {120, 110, 100}, {240, 240, 245}};
    int b = h < -150.0 ? 0 : h < 0.0 ? 1 : h < 150.0 ? 2 : h < 350.0 ? 3 : 4;
    return (uint32_t)c[b][0] | ((uint32_t)c[b][1] << 8) | ((uint32_t)c[b][2] << 16) | (255u << 24);
}

static uint64_t morton2(uint32_t x, uint32_t y) {
    uint64_t m = 0;
    for (int b = 0; b < 16; ++b)
        m |= ((uint64_t)((x >> b) & 1u) << (2 * b)) | ((uint64_t)((y >> b) & 1u) << (2 * b + 1));
    return m;
}

typedef struct { uint64_t code; int64_t cx, cz, start; } cell_t;
static int cell_cmp(const void* a, const void* b) {
    uint64_t x = ((const cell_t*)a)->code, y = ((const cell_t*)b)->code;
    return x < y ? -1 : x > y;
}

/*
 * Terrain scan: a jittered g x g grid on [0, extent]^2 in the x-z plane, height
 * y from the fBm above.  Points are stored cell by cell, cells of 64 x 64 grid
 * points ordered by Morton code, row-major inside a cell.  Record words:
 * RGBA8 from the height bands, intensity ~ U(0,1) as f32, zero padding.
 */
void nrvi_terrain(int64_t g, double extent, uint64_t seed, float* xyz, uint32_t* attr,
                  int64_t stride_words) {
    const int64_t C = 64;
    int64_t nc = (g + C - 1) / C;
    cell_t* cells = (cell_t*)malloc(sizeof(cell_t) * (size_t)(nc * nc));
    for (int64_t cz = 0; cz < nc; ++cz)
        for (int64_t cx = 0; cx < nc; ++cx) {
            cell_t* c = &cells[cz * nc + cx];
            c->code = morton2((uint32_t)cx, (uint32_t)cz); c->cx = cx; c->cz = cz;
        }
    qsort(cells, (size_t)(nc * nc), sizeof(cell_t), cell_cmp);
    int64_t run = 0;
    for (int64_t k = 0; k < nc * nc; ++k) {
        int64_t wx = g - C * cells[k].cx < C ? g - C * cells[k].cx : C;
        int64_t wz = g - C * cells[k].cz < C ? g - C * cells[k].cz : C;
        cells[k].start = run; run += wx * wz;
    }
    double sp = extent / (double)g;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < nc * nc; ++k) {
        int64_t cx = cells[k].cx, cz = cells[k].cz;
        int64_t wx = g - C * cx < C ? g - C * cx : C;
        int64_t wz = g - C * cz < C ? g - C * cz : C;
        for (int64_t b = 0; b < wz; ++b)
            for (int64_t a = 0; a < wx; ++a) {
                int64_t i = C * cx + a, j = C * cz + b, gi = j * g + i;
                int64_t o = cells[k].start + b * wx + a;
                double x = ((double)i + nrvi_uniform(seed, 0, (uint64_t)gi)) * sp;
                double z = ((double)j + nrvi_uniform(seed, 1, (uint64_t)gi)) * sp;
                double h = nrvi_terrain_height(seed, x, z);
                xyz[3 * o + 0] = (float)x; xyz[3 * o + 1] = (float)h; xyz[3 * o + 2] = (float)z;
                uint32_t* rec = attr + o * stride_words;
                rec[0] = nrvi_band_colour(h);
                rec[1] = f2u((float)nrvi_uniform(seed, 2, (uint64_t)gi));
                for (int64_t w = 2; w < stride_words; ++w) rec[w] = 0u;
            }
    }
    free(cells);
}

/*
 * Mean and standard deviation of one record channel over n records, in double.
 * fmt 0 = f32 word, 1 = u32 word, 2 = byte `comp` of a u8x4 word.  Summed in
 * fixed blocks of 2^16 records so the result does not depend on thread count.
 */
void nrvi_channel_moments(const uint32_t* attr, int64_t n, int64_t stride_words, int64_t word,
                          int fmt, int comp, double* mean, double* stdev) {
    const int64_t B = 65536;
    int64_t nb = (n + B - 1) / B;
    double* s1 = (double*)calloc((size_t)(nb > 0 ? nb : 1), sizeof(double));
    double* s2 = (double*)calloc((size_t)(nb > 0 ? nb : 1), sizeof(double));
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nb; ++b) {
        double a1 = 0.0, a2 = 0.0;
        int64_t e = (b + 1) * B < n ? (b + 1) * B : n;
        for (int64_t i = b * B; i < e; ++i) {
            uint32_t w = attr[i * stride_words + word];
            double v;
            if (fmt == 0) { float f; memcpy(&f, &w, 4); v = (double)f; }
            else if (fmt == 1) v = (double)w;
            else v = (double)((w >> (8 * comp)) & 255u);
            a1 += v; a2 += v * v;
        }
        s1[b] = a1; s2[b] = a2;
    }
    double t1 = 0.0, t2 = 0.0;
    for (int64_t b = 0; b < nb; ++b) { t1 += s1[b]; t2 += s2[b]; }
    free(s1); free(s2);
    double m = n > 0 ? t1 / (double)n : 0.0;
    double var = n > 0 ? t2 / (double)n - m * m : 0.0;
    *mean = m;
    *stdev = var > 0.0 ? sqrt(var) : 0.0;
}

/* Axis-aligned bounding box of n points (float -> exact in double). */
void nrvi_bbox(const float* xyz, int64_t n, double* lo, double* hi) {
    for (int j = 0; j < 3; ++j) { lo[j] = INFINITY; hi[j] = -INFINITY; }
    const int64_t B = 65536;
    int64_t nb = (n + B - 1) / B;
    double* part = (double*)malloc(sizeof(double) * 6 * (size_t)(nb > 0 ? nb : 1));
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nb; ++b) {
        double l[3] = {INFINITY, INFINITY, INFINITY}, h[3] = {-INFINITY, -INFINITY, -INFINITY};
        int64_t e = (b + 1) * B < n ? (b + 1) * B : n;
        for (int64_t i = b * B; i < e; ++i)
            for (int j = 0; j < 3; ++j) {
                double v = (double)xyz[3 * i + j];
                if (v < l[j]) l[j] = v;
                if (v > h[j]) h[j] = v;
            }
        for (int j = 0; j < 3; ++j) { part[6 * b + j] = l[j]; part[6 * b + 3 + j] = h[j]; }
    }
    for (int64_t b = 0; b < nb; ++b)
        for (int j = 0; j < 3; ++j) {
            if (part[6 * b + j] < lo[j]) lo[j] = part[6 * b + j];
            if (part[6 * b + 3 + j] > hi[j]) hi[j] = part[6 * b + 3 + j];
        }
    free(part);
}
