/*
 * Seeded synthetic chest-CT phantom: the input generator shared by the CPU
 * oracle's tests and the GPU path's tests and benchmark.
 *
 * This module holds no arithmetic of the segmentation method (no histogram,
 * no entropy, no threshold). It only maps (seed, volume id, z, y, x) to an
 * int16 Hounsfield value, with integer arithmetic only, so that the host build
 * (gcc) and the device build (nvcc) produce bit-identical volumes.
 *
 * Geometry (all integer, image units scaled to the slice size):
 *   outside air   : mu = -1024, no class spread
 *   body ellipse  : mu = body_mu, sd = body_sd
 *   two lungs     : mu = lung_mu, sd = lung_sd
 *   airway capsules (a tree of line segments with radius; a disc when the
 *   segment is a point in one slice): mu = air_mu, sd = air_sd
 * plus sensor noise of sd noise_sd on every voxel.
 *
 * Gaussian draws: Irwin-Hall sum of twelve 16-bit uniforms taken from three
 * SplitMix64 outputs (Steele, Lea & Flood 2014; the 64-bit finaliser published
 * by Vigna), centred and scaled in fixed point, so the value is an integer.
 */
#ifndef PHANTOM_H
#define PHANTOM_H

#include <stdint.h>

#ifdef __CUDACC__
#define PH_HD __host__ __device__ __forceinline__
#else
#define PH_HD static inline
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Capsule: segment a->b with radius r, all in 1/16-voxel fixed point. */
typedef struct {
    int32_t ax, ay, az, bx, by, bz, r;
    int32_t zlo, zhi; /* slice range the capsule can touch (inclusive) */
    int32_t ylo, yhi, xlo, xhi; /* voxel bounding box */
} ph_capsule;

typedef struct {
    int32_t cx, cy, a, b; /* centre and semi-axes in voxels */
} ph_ellipse;

typedef struct {
    int64_t nx, ny, nz;
    uint64_t seed;
    uint32_t vol_id;
    int32_t air_hu;         /* outside air value, -1024 */
    int32_t body_mu, body_sd;
    int32_t lung_mu, lung_sd;
    int32_t airway_mu, airway_sd;
    int32_t noise_sd;
    ph_ellipse body, lung[2];
    int32_t ncaps;
    const ph_capsule* caps;     /* host or device pointer, per build */
    const int32_t* slice_off;   /* [nz+1] CSR offsets into slice_caps */
    const int32_t* slice_caps;  /* capsule indices touching each slice */
} ph_desc;

enum { PH_AIR = 0, PH_BODY = 1, PH_LUNG = 2, PH_AIRWAY = 3 };

PH_HD uint64_t ph_splitmix64(uint64_t state) {
    uint64_t z = state + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Irwin-Hall approximation of sd * N(0,1), rounded to an integer.
 * counter identifies the draw; three hash outputs give 12 uniforms. */
PH_HD int32_t ph_gauss(uint64_t seed, uint64_t counter, int32_t sd) {
    if (sd == 0) return 0;
    int64_t s = 0;
    for (int k = 0; k < 3; ++k) {
        uint64_t h = ph_splitmix64(seed ^ (counter * 4ull + (uint64_t)k) * 0xD1B54A32D192ED03ull);
        s += (int64_t)(h & 0xFFFF) + (int64_t)((h >> 16) & 0xFFFF) +
             (int64_t)((h >> 32) & 0xFFFF) + (int64_t)(h >> 48);
    }
    /* mean of the sum is 12 * 65535 / 2 = 393210; sd is about 65535 */
    int64_t c = 2 * s - 786420;                 /* 2 * (s - mean), exact */
    int64_t num = (int64_t)sd * c + 65536;      /* round to nearest */
    /* floor division by 131072 that does not depend on signed shifts */
    int64_t q = num >= 0 ? num / 131072 : -((-num + 131071) / 131072);
    return (int32_t)q;
}

PH_HD int ph_in_ellipse(const ph_ellipse* e, int64_t x, int64_t y) {
    int64_t dx = x - e->cx, dy = y - e->cy;
    int64_t a2 = (int64_t)e->a * e->a, b2 = (int64_t)e->b * e->b;
    return dx * dx * b2 + dy * dy * a2 <= a2 * b2;
}

/* Exact integer test: distance from voxel centre p to segment ab <= r. */
PH_HD int ph_in_capsule(const ph_capsule* c, int64_t x, int64_t y, int64_t z) {
    int64_t px = x * 16 + 8, py = y * 16 + 8, pz = z * 16 + 8;
    int64_t ex = c->bx - c->ax, ey = c->by - c->ay, ez = c->bz - c->az;
    int64_t dx = px - c->ax, dy = py - c->ay, dz = pz - c->az;
    int64_t r2 = (int64_t)c->r * c->r;
    int64_t den = ex * ex + ey * ey + ez * ez;
    int64_t tn = dx * ex + dy * ey + dz * ez;
    int64_t d2 = dx * dx + dy * dy + dz * dz;
    if (den == 0 || tn <= 0) return d2 <= r2;
    if (tn >= den) {
        int64_t fx = px - c->bx, fy = py - c->by, fz = pz - c->bz;
        return fx * fx + fy * fy + fz * fz <= r2;
    }
    /* perpendicular distance^2 * den = d2 * den - tn^2 (exact in int64 for
     * coordinates below 2^14 voxels * 16) */
    return d2 * den - tn * tn <= r2 * den;
}

PH_HD int ph_class(const ph_desc* d, int64_t z, int64_t y, int64_t x) {
    int cls = PH_AIR;
    if (ph_in_ellipse(&d->body, x, y)) cls = PH_BODY;
    if (ph_in_ellipse(&d->lung[0], x, y) || ph_in_ellipse(&d->lung[1], x, y)) cls = PH_LUNG;
    if (d->ncaps > 0) {
        int32_t b = d->slice_off[z], e = d->slice_off[z + 1];
        for (int32_t k = b; k < e; ++k) {
            const ph_capsule* c = &d->caps[d->slice_caps[k]];
            if (y < c->ylo || y > c->yhi || x < c->xlo || x > c->xhi) continue;
            if (ph_in_capsule(c, x, y, z)) { cls = PH_AIRWAY; break; }
        }
    }
    return cls;
}

PH_HD int16_t ph_voxel(const ph_desc* d, int64_t z, int64_t y, int64_t x) {
    int cls = ph_class(d, z, y, x);
    int32_t mu = d->air_hu, sd = 0;
    if (cls == PH_BODY) { mu = d->body_mu; sd = d->body_sd; }
    else if (cls == PH_LUNG) { mu = d->lung_mu; sd = d->lung_sd; }
    else if (cls == PH_AIRWAY) { mu = d->airway_mu; sd = d->airway_sd; }
    uint64_t idx = (((uint64_t)d->vol_id * 65536ull + (uint64_t)z) * 65536ull + (uint64_t)y) * 65536ull + (uint64_t)x;
    int32_t v = mu + ph_gauss(d->seed, idx * 2ull, sd) + ph_gauss(d->seed, idx * 2ull + 1ull, d->noise_sd);
    if (v < -32768) v = -32768;
    if (v > 32767) v = 32767;
    return (int16_t)v;
}

/* Host generator: fills out[nz][ny][nx] using nthreads host threads. */
int ph_generate_host(const ph_desc* d, int16_t* out, int nthreads);

#ifdef __cplusplus
}
#endif
#endif /* PHANTOM_H */
