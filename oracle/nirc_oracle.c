/*
 * nirc_oracle.c -- plain CPU oracle of the Neural Incident Radiance Cache
 * (NIRC) two-level Monte Carlo hot path (arXiv 2412.04634).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * definition the CUDA kernels are checked against.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg load it; the product
 * library never links, calls or falls back to it.  It shares no code,
 * header, table or helper with the CUDA path: both read the same seeded
 * input blobs (scene, parameters, records) and each implements the
 * counter-based generator Philox4x32-10 from its published definition.
 *
 * Precision: continuous quantities (encodings, network, BSDF weights,
 * radiance, estimator sums, loss, gradients, Adam) are FP64.  Quantities
 * that decide an integer -- ray/primitive intersection, hit points, sampled
 * directions, disk-rejection tests, Russian-roulette tests and hash-grid
 * cells -- are computed in strict IEEE binary32 in a fixed operation order
 * (compile with -ffp-contract=off, no fast-math), the precision the GPU path
 * takes these decisions in, so both sides make the same decisions.
 *
 * Light modes (eq. Lsplit): mode 0 caches the full incident radiance and
 * traces pure BSDF paths; mode 1 splits L_i = L_ind + L_nee, estimates the
 * direct part by next-event estimation on rectangular emitters combined
 * with BSDF sampling by the power heuristic (at the shading point the M
 * residual directions are the BSDF technique, along a path the continuation
 * direction), and the cache, the residual paths and the training targets
 * carry L_ind (the emission of a path's first hit belongs to L_nee).
 *
 * Parity pins (tests/test_oracle_*.py): Philox against a library
 * implementation and its published known answer; the white-furnace closed
 * form (constant cache on a Lambertian surface gives rho*L per sample); the
 * furnace path expectation L_e * sum_k rho^k; zero cache == plain path
 * tracing; analytic cache gives a residual of zero mean; unbiasedness of the
 * two-level estimator; the network against a library MLP; encodings and
 * hash indices against closed forms and hand-computed values; gradients
 * against central finite differences; Adam against its closed-form first
 * steps; MRSE against closed forms.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define O_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Input layouts (the seeded generator's binary formats)                    */
/* ------------------------------------------------------------------------ */

typedef struct {
    float a[3];
    float radius;
    float u[3];
    float inv_uu;
    float v[3];
    float inv_vv;
    float n[3];
    uint32_t kind; /* 0 sphere, 1 rectangle */
    float albedo[3];
    float roughness;
    float emission[3];
    uint32_t flags; /* bits 0-1 material, bit 8 two-sided emission */
} o_prim;

typedef struct {
    uint32_t n_prims;
    uint32_t pad[3];
    float origin[4];
    float top_left[4];
    float horizontal[4];
    float vertical[4];
    uint32_t reserved[4];
} o_header;

typedef struct {
    float p[3];
    float n[3];
    float wo[3];
    float albedo[3];
    float roughness;
    uint32_t prim;
    uint32_t flags; /* bit 0 valid, bits 1-2 material */
    uint32_t pad;
} o_record;

typedef struct {
    int32_t pos_encoding; /* 0 frequency encoding of x, 1 hash grid */
    int32_t hash_levels;
    int32_t feats_per_level;
    int32_t log2_table;
    int32_t base_res;
    int32_t freq_octaves;
    int32_t width;
    int32_t hidden_layers;
    int32_t input_encoding; /* 0 frequency encodings of w and n, 1 the paper's (spherical harmonics + phi) */
    int32_t output;         /* 0 radiance: n = exp(z), relative L2 loss; 1 visibility: V = sigmoid(z), L2 loss */
    double growth;
    double z_clamp;
    double loss_eps;
} o_cfg;

typedef struct {
    uint32_t width, height;
    uint32_t n_cache;   /* N: cache-level samples per pixel */
    uint32_t n_resid;   /* M: residual-level samples per pixel */
    uint32_t max_depth; /* segments of a residual path */
    uint32_t frame;
    uint64_t seed;
    uint32_t cache_mode; /* 0 network, 1 zero, 2 constant */
    uint32_t light_mode; /* 0 cache = full L_i, 1 cache = L_ind with NEE + MIS (eq. Lsplit) */
    uint32_t estimator;  /* 0 two-level (eq. L_mlmc), 1 biased with the Balanced Termination Heuristic,
                            2 two-level at the first three vertices of each path */
    uint32_t n_cache2;   /* estimator 2: cache samples at the second and third vertex */
    uint32_t n_cache3;
    double cache_const[3];
} o_frame;

enum { MAT_LAMBERT = 0, MAT_GGX = 1, MAT_BLACK = 2 };
enum { KIND_SPHERE = 0, KIND_RECT = 1 };
enum { EMIT_TWO_SIDED = 1u << 8 };

/* Philox counter word 3: what a draw is for (see the header of this file
 * and the CUDA path's documentation; the same table is restated there). */
enum {
    PURPOSE_CAMERA = 1,
    PURPOSE_CACHE_DIR = 2,
    PURPOSE_RESID_DIR = 3,
    PURPOSE_BOUNCE = 4, /* + 16 * segment */
    PURPOSE_RR = 5,     /* + 16 * segment */
    PURPOSE_TRAIN_PICK = 6,
    PURPOSE_LIGHT = 7,  /* + 16 * segment (0: the shading point) */
    PURPOSE_BTH_DIR = 8, /* + 16 * vertex: the scattering direction sampled at a biased path's vertex */
    PURPOSE_BTH_XI = 9,  /* + 16 * vertex: the termination test's uniform */
    PURPOSE_VCACHE = 10  /* + 16 * vertex (2, 3): cache samples at later vertices of a residual path */
};

static const float T_MIN = 1e-4f;
static const float RR_CONTINUE = 0.9f; /* Russian roulette: terminate with probability 0.1 */
static const double F0_SPEC = 0.04;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)                         */
/* ------------------------------------------------------------------------ */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += 0x9E3779B9u; /* golden ratio */
            k1 += 0xBB67AE85u; /* sqrt(3) - 1 */
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

static void philox(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                   uint32_t out[4])
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {k0, k1};
    orc_philox4x32_10(ctr, key, out);
}

/* 24 high bits of a word -> float in [0, 1), exact in binary32. */
static float u01(uint32_t x)
{
    return (float)(x >> 8) * (1.0f / 16777216.0f);
}

/* 64-bit FNV-1a over 32-bit words: path signature of discrete decisions. */
static uint64_t sig_mix(uint64_t h, uint32_t word)
{
    h ^= (uint64_t)word;
    h *= 0x100000001B3ull;
    return h;
}
#define SIG_INIT 0xCBF29CE484222325ull

/* ------------------------------------------------------------------------ */
/* Strict binary32 geometry (decides hits, hit points and directions)       */
/* ------------------------------------------------------------------------ */

static float dot3f(const float a[3], const float b[3])
{
    float xy = a[0] * b[0] + a[1] * b[1];
    return xy + a[2] * b[2];
}

static void normalize3f(float v[3])
{
    float len = sqrtf(dot3f(v, v));
    float inv = 1.0f / len;
    v[0] = v[0] * inv;
    v[1] = v[1] * inv;
    v[2] = v[2] * inv;
}

static int hit_sphere(const o_prim* s, const float o[3], const float d[3], float* t_out)
{
    float oc[3] = {o[0] - s->a[0], o[1] - s->a[1], o[2] - s->a[2]};
    float b = dot3f(oc, d);
    float c = dot3f(oc, oc) - s->radius * s->radius;
    float disc = b * b - c;
    if (!(disc >= 0.0f)) return 0;
    float sq = sqrtf(disc);
    float t0 = -b - sq;
    float t1 = -b + sq;
    if (t0 > T_MIN) {
        *t_out = t0;
        return 1;
    }
    if (t1 > T_MIN) {
        *t_out = t1;
        return 1;
    }
    return 0;
}

static int hit_rect(const o_prim* r, const float o[3], const float d[3], float* t_out)
{
    float denom = dot3f(r->n, d);
    if (denom == 0.0f) return 0;
    float ao[3] = {r->a[0] - o[0], r->a[1] - o[1], r->a[2] - o[2]};
    float t = dot3f(r->n, ao) / denom;
    if (!(t > T_MIN)) return 0;
    float p[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
    float rel[3] = {p[0] - r->a[0], p[1] - r->a[1], p[2] - r->a[2]};
    float al = dot3f(rel, r->u) * r->inv_uu;
    float be = dot3f(rel, r->v) * r->inv_vv;
    if (!(al >= 0.0f && al <= 1.0f && be >= 0.0f && be <= 1.0f)) return 0;
    *t_out = t;
    return 1;
}

/* Nearest hit along o + t d, t > T_MIN; ties go to the lower index. */
static int trace_nearest(const o_prim* prims, uint32_t n_prims, const float o[3], const float d[3],
                         float* t_hit)
{
    float best = INFINITY;
    int idx = -1;
    for (uint32_t i = 0; i < n_prims; i++) {
        float t;
        int hit = prims[i].kind == KIND_SPHERE ? hit_sphere(&prims[i], o, d, &t)
                                               : hit_rect(&prims[i], o, d, &t);
        if (hit && t < best) {
            best = t;
            idx = (int)i;
        }
    }
    *t_hit = best;
    return idx;
}

typedef struct {
    float p[3];
    float n[3];     /* unit normal facing the incoming ray */
    int front;      /* ray arrives on the side the stored normal points to */
} o_hit;

static void hit_info(const o_prim* pr, const float o[3], const float d[3], float t, o_hit* h)
{
    h->p[0] = o[0] + t * d[0];
    h->p[1] = o[1] + t * d[1];
    h->p[2] = o[2] + t * d[2];
    float n[3];
    if (pr->kind == KIND_SPHERE) {
        n[0] = h->p[0] - pr->a[0];
        n[1] = h->p[1] - pr->a[1];
        n[2] = h->p[2] - pr->a[2];
        normalize3f(n);
    } else {
        n[0] = pr->n[0];
        n[1] = pr->n[1];
        n[2] = pr->n[2];
    }
    float dn = dot3f(n, d);
    h->front = dn < 0.0f;
    if (dn > 0.0f) {
        n[0] = -n[0];
        n[1] = -n[1];
        n[2] = -n[2];
    }
    h->n[0] = n[0];
    h->n[1] = n[1];
    h->n[2] = n[2];
}

/* Emitted radiance L_e(y, -d) of a hit primitive (one- or two-sided). */
static void emitted(const o_prim* pr, int front, double le[3])
{
    int on = front || (pr->flags & EMIT_TWO_SIDED);
    for (int c = 0; c < 3; c++) le[c] = on ? (double)pr->emission[c] : 0.0;
}

/* ------------------------------------------------------------------------ */
/* BSDF sampling (independent BSDF importance sampling for L_c and L_r)     */
/* ------------------------------------------------------------------------ */

/* Orthonormal basis around unit n (Duff et al., JCGT 2017). */
static void onb(const float n[3], float t[3], float b[3])
{
    float sign = copysignf(1.0f, n[2]);
    float a = -1.0f / (sign + n[2]);
    float bb = (n[0] * n[1]) * a;
    t[0] = 1.0f + ((sign * n[0]) * n[0]) * a;
    t[1] = sign * bb;
    t[2] = (-sign) * n[0];
    b[0] = bb;
    b[1] = sign + (n[1] * n[1]) * a;
    b[2] = -n[1];
}

/* Uniform point on the unit disk by rejection from the square: up to 8
 * Philox calls (counter word 2 = call index), two candidates per call.
 * Returns the number of rejected candidates (16 = gave up, point (0, 0)). */
static uint32_t disk_sample(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c3, float* a,
                            float* b)
{
    uint32_t rejected = 0;
    for (uint32_t call = 0; call < 8; call++) {
        uint32_t r[4];
        philox(k0, k1, c0, c1, call, c3, r);
        for (int j = 0; j < 4; j += 2) {
            float x = 2.0f * u01(r[j]) - 1.0f;
            float y = 2.0f * u01(r[j + 1]) - 1.0f;
            float s = x * x + y * y;
            if (s < 1.0f) {
                *a = x;
                *b = y;
                return rejected;
            }
            rejected++;
        }
    }
    *a = 0.0f;
    *b = 0.0f;
    return rejected;
}

static void to_world(float lx, float ly, float lz, const float t[3], const float b[3], const float n[3],
                     float w[3])
{
    for (int k = 0; k < 3; k++) w[k] = (lx * t[k] + ly * b[k]) + lz * n[k];
}

/* GGX visible-normal sample (Heitz, JCGT 2018) with the disk point (t1, t2);
 * returns the reflected direction in world space. */
static void ggx_vndf_reflect(const float wo[3], const float t[3], const float b[3], const float n[3],
                             float alpha, float t1, float t2, float wi[3])
{
    float wl[3] = {dot3f(wo, t), dot3f(wo, b), dot3f(wo, n)};
    float vh[3] = {alpha * wl[0], alpha * wl[1], wl[2]};
    normalize3f(vh);
    float lensq = vh[0] * vh[0] + vh[1] * vh[1];
    float T1[3];
    if (lensq > 0.0f) {
        float il = 1.0f / sqrtf(lensq);
        T1[0] = (-vh[1]) * il;
        T1[1] = vh[0] * il;
        T1[2] = 0.0f;
    } else {
        T1[0] = 1.0f;
        T1[1] = 0.0f;
        T1[2] = 0.0f;
    }
    float T2[3] = {vh[1] * T1[2] - vh[2] * T1[1], vh[2] * T1[0] - vh[0] * T1[2],
                   vh[0] * T1[1] - vh[1] * T1[0]};
    float s = 0.5f * (1.0f + vh[2]);
    float t2w = (1.0f - s) * sqrtf(1.0f - t1 * t1) + s * t2;
    float nz = sqrtf(fmaxf(0.0f, (1.0f - t1 * t1) - t2w * t2w));
    float nh[3];
    for (int k = 0; k < 3; k++) nh[k] = (t1 * T1[k] + t2w * T2[k]) + nz * vh[k];
    float ne[3] = {alpha * nh[0], alpha * nh[1], fmaxf(0.0f, nh[2])};
    normalize3f(ne);
    float h[3];
    to_world(ne[0], ne[1], ne[2], t, b, n, h);
    float dh = dot3f(wo, h);
    float two_dh = 2.0f * dh;
    for (int k = 0; k < 3; k++) wi[k] = two_dh * h[k] - wo[k];
    normalize3f(wi);
}

static double dot3d(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* GGX denominator dd = 1 - cos^2 (1 - a2) = sin^2 + a2 cos^2 of the angle
 * between n and h, from the cross and dot products normalised by the
 * vectors' lengths: no cancellation near the specular peak and no
 * dependence on the binary32 rounding of the stored unit normal (which
 * would move 1 - cos^2 by ~1e-7, a large relative change of dd at small
 * roughness). */
static double ggx_dd(const double n[3], const double h[3], double a2)
{
    double c[3] = {n[1] * h[2] - n[2] * h[1], n[2] * h[0] - n[0] * h[2], n[0] * h[1] - n[1] * h[0]};
    double nh = dot3d(n, h);
    double norm = dot3d(n, n) * dot3d(h, h);
    return (dot3d(c, c) + a2 * nh * nh) / norm;
}

/* f_r(x, wi, wo) cos(theta_i) / p(wi) of the Lambertian + GGX material with
 * the one-sample mixture (1/2 cosine, 1/2 GGX visible normals), FP64. */
static void ggx_mix_weight(const o_record* rec, const float wif[3], double w[3])
{
    double n[3] = {rec->n[0], rec->n[1], rec->n[2]};
    double wo[3] = {rec->wo[0], rec->wo[1], rec->wo[2]};
    double wi[3] = {wif[0], wif[1], wif[2]};
    double alpha = (double)(rec->roughness * rec->roughness);
    double a2 = alpha * alpha;
    double ci = dot3d(n, wi), co = dot3d(n, wo);
    double h[3] = {wo[0] + wi[0], wo[1] + wi[1], wo[2] + wi[2]};
    double hl = sqrt(dot3d(h, h));
    for (int k = 0; k < 3; k++) h[k] /= hl;
    double oh = dot3d(wo, h);
    if (oh < 0.0) oh = 0.0;
    if (oh > 1.0) oh = 1.0;
    double dd = ggx_dd(n, h, a2);
    double D = a2 / (O_PI * dd * dd);
    double lam_o = sqrt(a2 + (1.0 - a2) * co * co);
    double lam_i = sqrt(a2 + (1.0 - a2) * ci * ci);
    double G2 = 2.0 * ci * co / (co * lam_i + ci * lam_o);
    double G1o = 2.0 * co / (co + lam_o);
    double F = F0_SPEC + (1.0 - F0_SPEC) * pow(1.0 - oh, 5.0);
    double fs = F * D * G2 / (4.0 * ci * co);
    double pdf_s = G1o * D / (4.0 * co);
    double pdf = 0.5 * ci / O_PI + 0.5 * pdf_s;
    for (int c = 0; c < 3; c++) w[c] = ((double)rec->albedo[c] / O_PI + fs) * ci / pdf;
}

typedef struct {
    float wi[3];
    double w[3];    /* f_r cos / p, zero when invalid */
    int valid;      /* direction above the surface and material scatters */
    uint32_t rejected;
    uint32_t lobe;  /* 0 cosine, 1 GGX */
} o_sample;

static uint32_t sample_word(const o_sample* s)
{
    return s->rejected | (s->lobe << 8) | ((uint32_t)s->valid << 9);
}

/* BSDF importance sample at a shading record; Philox counter
 * (c0, c1, call, c3).  The lobe choice uses the low byte of call 0, word 0. */
static void sample_bsdf(const o_record* rec, uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c3,
                        o_sample* out)
{
    uint32_t mat = (rec->flags >> 1) & 3u;
    memset(out, 0, sizeof(*out));
    if (mat == MAT_BLACK) {
        out->wi[0] = rec->n[0];
        out->wi[1] = rec->n[1];
        out->wi[2] = rec->n[2];
        return;
    }
    float t[3], b[3];
    onb(rec->n, t, b);
    if (mat == MAT_GGX) {
        /* mixture lobe: low byte of word 0 of the first Philox call (the disk
         * candidates use only the high 24 bits of each word) */
        uint32_t r[4];
        philox(k0, k1, c0, c1, 0u, c3, r);
        out->lobe = (r[0] & 0xFFu) < 128u ? 0u : 1u;
    }
    float da, db;
    out->rejected = disk_sample(k0, k1, c0, c1, c3, &da, &db);
    if (out->lobe == 0) {
        float s = da * da + db * db;
        float z = sqrtf(fmaxf(0.0f, 1.0f - s));
        to_world(da, db, z, t, b, rec->n, out->wi);
        normalize3f(out->wi);
    } else {
        float alpha = rec->roughness * rec->roughness;
        ggx_vndf_reflect(rec->wo, t, b, rec->n, alpha, da, db, out->wi);
    }
    if (!(dot3f(out->wi, rec->n) > 0.0f)) return; /* below the surface: weight 0 */
    out->valid = 1;
    if (mat == MAT_LAMBERT) {
        /* (rho / pi) cos / (cos / pi) = rho */
        for (int c = 0; c < 3; c++) out->w[c] = (double)rec->albedo[c];
    } else {
        ggx_mix_weight(rec, out->wi, out->w);
    }
}

/* ------------------------------------------------------------------------ */
/* Encodings: frequency (sin/cos octaves) and multiresolution hash grid      */
/* ------------------------------------------------------------------------ */

static int n_pos_features(const o_cfg* c)
{
    return c->pos_encoding == 1 ? c->hash_levels * c->feats_per_level : 3 * 2 * c->freq_octaves;
}

#define SH_COEFFS 25   /* real spherical harmonics of degree l = 0..4 */
#define BLOB_BINS 4    /* one-blob bins of each phi scalar */
#define PHI_FEATURES (3 + 2 * BLOB_BINS + BLOB_BINS)

static int n_dir_features(const o_cfg* c)
{
    return c->input_encoding == 1 ? SH_COEFFS : 2 * 2 * c->freq_octaves;
}

static int n_surface_features(const o_cfg* c)
{
    return c->input_encoding == 1 ? PHI_FEATURES : 3 * 2 * c->freq_octaves;
}

static int n_inputs(const o_cfg* c)
{
    return n_pos_features(c) + n_dir_features(c) + n_surface_features(c);
}

/* sin(2^k pi v), cos(2^k pi v), k = 0..octaves-1 */
static int freq_encode(double v, int octaves, double* e)
{
    for (int k = 0; k < octaves; k++) {
        double arg = O_PI * ldexp(v, k);
        e[2 * k] = sin(arg);
        e[2 * k + 1] = cos(arg);
    }
    return 2 * octaves;
}

/* theta_hat = theta / pi and phi_hat = phi / (2 pi) in [0, 1) of a unit
 * vector (polar angle from +z, azimuth from +x towards +y). */
static void unit_angles(const float w[3], double* theta_hat, double* phi_hat)
{
    double wz = (double)w[2];
    if (wz > 1.0) wz = 1.0;
    if (wz < -1.0) wz = -1.0;
    *theta_hat = acos(wz) / O_PI;
    double ph = atan2((double)w[1], (double)w[0]) / (2.0 * O_PI);
    if (ph < 0.0) ph += 1.0;
    *phi_hat = ph;
}

static double factorial(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; i++) f *= i;
    return f;
}

/* Real spherical harmonics Y_l^m, l = 0..4, of the direction of w (paper,
 * section "Neural Network Architecture": spherical-harmonics coefficients of
 * w_i, 25 values per request), orthonormal on the unit sphere, stored at
 * index l*l + l + m:
 *   Y_l^0  = K_l^0 P_l^0(cos t)
 *   Y_l^m  = sqrt(2) K_l^m P_l^m(cos t) cos(m p)   (m > 0)
 *   Y_l^-m = sqrt(2) K_l^m P_l^m(cos t) sin(m p)   (m > 0)
 * with K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), (t, p) the polar angle and
 * azimuth of w, and P_l^m the associated Legendre functions without the
 * Condon-Shortley phase, from the textbook recurrences
 *   P_m^m = (2m-1)!! sin^m t,  P_{m+1}^m = (2m+1) cos t P_m^m,
 *   (l-m) P_l^m = (2l-1) cos t P_{l-1}^m - (l+m-1) P_{l-2}^m. */
void orc_sh_basis(const float w[3], double* e)
{
    double x = w[0], y = w[1], z = w[2];
    double r = sqrt(x * x + y * y + z * z);
    double ct = z / r, st = sqrt(x * x + y * y) / r;
    double ph = atan2(y, x);
    double P[5][5];
    for (int m = 0; m <= 4; m++) {
        double pmm = 1.0;
        for (int i = 1; i <= m; i++) pmm *= (2.0 * i - 1.0) * st;
        P[m][m] = pmm;
        if (m + 1 <= 4) P[m + 1][m] = (2.0 * m + 1.0) * ct * pmm;
        for (int l = m + 2; l <= 4; l++)
            P[l][m] = ((2.0 * l - 1.0) * ct * P[l - 1][m] - (l + m - 1.0) * P[l - 2][m]) / (l - m);
    }
    for (int l = 0; l <= 4; l++) {
        for (int m = 0; m <= l; m++) {
            double K = sqrt((2.0 * l + 1.0) / (4.0 * O_PI) * factorial(l - m) / factorial(l + m));
            if (m == 0) {
                e[l * l + l] = K * P[l][0];
            } else {
                e[l * l + l + m] = sqrt(2.0) * K * P[l][m] * cos(m * ph);
                e[l * l + l - m] = sqrt(2.0) * K * P[l][m] * sin(m * ph);
            }
        }
    }
}

/* One-blob encoding of s in [0, 1] into k bins (Mueller et al. 2019, the
 * encoding NRC gives these inputs): a Gaussian kernel of standard deviation
 * 1/k centred at s, integrated over each bin [i/k, (i+1)/k):
 *   e_i = G((i+1)/k - s) - G(i/k - s),  G(u) = (1 + erf(u k / sqrt 2)) / 2,
 * with no wrap-around at the ends. */
void orc_one_blob(double s, int k, double* e)
{
    double scale = k / sqrt(2.0);
    for (int i = 0; i < k; i++) {
        double lo = (double)i / k - s, hi = (double)(i + 1) / k - s;
        e[i] = 0.5 * (erf(hi * scale) - erf(lo * scale));
    }
}

/* The per-surface inputs phi of the paper's encoding (paper: shading normal,
 * albedo and roughness fed with NRC's encodings): albedo as is (3), the
 * normal's (theta_hat, phi_hat) one-blob encoded (2 x 4) and the roughness
 * one-blob encoded (4). */
static void phi_encode(const o_record* rec, double* e)
{
    for (int k = 0; k < 3; k++) e[k] = (double)rec->albedo[k];
    double th, ph;
    unit_angles(rec->n, &th, &ph);
    orc_one_blob(th, BLOB_BINS, e + 3);
    orc_one_blob(ph, BLOB_BINS, e + 3 + BLOB_BINS);
    orc_one_blob((double)rec->roughness, BLOB_BINS, e + 3 + 2 * BLOB_BINS);
}

static uint32_t grid_resolution(const o_cfg* c, int level)
{
    return (uint32_t)floor((double)c->base_res * pow(c->growth, (double)level));
}

/* Level l of the hash grid: the 8 cell-corner table indices and trilinear
 * weights of position x (InstantNGP).  Cells are found in binary32. */
void orc_hash_level(const o_cfg* c, int level, const float x[3], uint32_t idx[8], double wts[8])
{
    uint32_t res = grid_resolution(c, level);
    uint64_t T = 1ull << c->log2_table;
    uint64_t side = (uint64_t)res + 1;
    int dense = side * side * side <= T;
    float fres = (float)res;
    uint32_t cell[3];
    float frac[3];
    for (int d = 0; d < 3; d++) {
        float xc = fminf(fmaxf(x[d], 0.0f), 1.0f);
        float ps = xc * fres;
        float fl = floorf(ps);
        if (fl >= fres) fl = fres - 1.0f;
        cell[d] = (uint32_t)fl;
        frac[d] = ps - fl;
    }
    for (int corner = 0; corner < 8; corner++) {
        uint32_t v[3];
        double w = 1.0;
        for (int d = 0; d < 3; d++) {
            uint32_t bit = (corner >> d) & 1u;
            v[d] = cell[d] + bit;
            w *= bit ? (double)frac[d] : 1.0 - (double)frac[d];
        }
        uint64_t index;
        if (dense) {
            index = (uint64_t)v[0] + (uint64_t)v[1] * side + (uint64_t)v[2] * side * side;
        } else {
            uint32_t hsh = (v[0] * 1u) ^ (v[1] * 2654435761u) ^ (v[2] * 805459861u);
            index = (uint64_t)(hsh & (uint32_t)(T - 1));
        }
        idx[corner] = (uint32_t)index;
        wts[corner] = w;
    }
}

/* Network input for the shading record rec and incident direction w:
 * [position features][direction features][surface features].
 * input_encoding 0: direction = frequency encoding of (theta_hat, phi_hat),
 *   surface = frequency encoding of the normal's three components;
 * input_encoding 1 (the paper's): direction = the 25 spherical-harmonics
 *   values of w, surface = phi (albedo, normal and roughness). */
static void encode(const o_cfg* c, const double* hash_table, const o_record* rec, const float w[3], double* e)
{
    int k = 0;
    const float* p = rec->p;
    if (c->pos_encoding == 1) {
        uint64_t T = 1ull << c->log2_table;
        int F = c->feats_per_level;
        for (int l = 0; l < c->hash_levels; l++) {
            uint32_t idx[8];
            double wts[8];
            orc_hash_level(c, l, p, idx, wts);
            const double* tab = hash_table + (uint64_t)l * T * F;
            for (int f = 0; f < F; f++) {
                double acc = 0.0;
                for (int corner = 0; corner < 8; corner++) acc += wts[corner] * tab[(uint64_t)idx[corner] * F + f];
                e[k++] = acc;
            }
        }
    } else {
        for (int d = 0; d < 3; d++) k += freq_encode((double)p[d], c->freq_octaves, e + k);
    }
    if (c->input_encoding == 1) {
        orc_sh_basis(w, e + k);
        phi_encode(rec, e + k + SH_COEFFS);
        return;
    }
    double theta_hat, phi_hat;
    unit_angles(w, &theta_hat, &phi_hat);
    k += freq_encode(theta_hat, c->freq_octaves, e + k);
    k += freq_encode(phi_hat, c->freq_octaves, e + k);
    for (int d = 0; d < 3; d++) k += freq_encode((double)rec->n[d], c->freq_octaves, e + k);
}

/* ------------------------------------------------------------------------ */
/* The network n_i(x, w_i, phi; w): ReLU MLP with biases, exp output         */
/* ------------------------------------------------------------------------ */

#define MAX_WIDTH 256
#define MAX_LAYERS 16

static uint64_t mlp_param_count(const o_cfg* c)
{
    uint64_t n = 0;
    int in = n_inputs(c);
    for (int l = 0; l <= c->hidden_layers; l++) {
        int out = l == c->hidden_layers ? 3 : c->width;
        n += (uint64_t)out * in + out;
        in = out;
    }
    return n;
}

uint64_t orc_param_count(const o_cfg* c)
{
    uint64_t n = mlp_param_count(c);
    if (c->pos_encoding == 1) n += (uint64_t)c->hash_levels * (1ull << c->log2_table) * c->feats_per_level;
    return n;
}

/* Forward pass.  pre[l][j] / act[l][j] (optional) receive the hidden
 * pre-activations and ReLU outputs; z receives the three output logits. */
static void mlp_forward(const o_cfg* c, const double* params, const double* e, double* pre, double* act,
                        double z[3])
{
    double buf_in[MAX_WIDTH * 2], buf_out[MAX_WIDTH];
    int in = n_inputs(c);
    const double* x = e;
    const double* P = params;
    for (int l = 0; l <= c->hidden_layers; l++) {
        int out = l == c->hidden_layers ? 3 : c->width;
        const double* W = P;
        const double* b = P + (uint64_t)out * in;
        for (int o = 0; o < out; o++) {
            double s = b[o];
            for (int i = 0; i < in; i++) s += W[(uint64_t)o * in + i] * x[i];
            buf_out[o] = s;
        }
        P += (uint64_t)out * in + out;
        if (l == c->hidden_layers) {
            for (int o = 0; o < 3; o++) z[o] = buf_out[o];
        } else {
            for (int o = 0; o < out; o++) {
                if (pre) pre[l * MAX_WIDTH + o] = buf_out[o];
                buf_in[o] = buf_out[o] > 0.0 ? buf_out[o] : 0.0;
                if (act) act[l * MAX_WIDTH + o] = buf_in[o];
            }
            x = buf_in;
            in = out;
        }
    }
}

/* Output activation: radiance n = exp(min(z, z_clamp)); visibility (the
 * Neural Visibility Cache, paper section "Neural Visibility Cache": a
 * sigmoid on the output neurons) V = 1 / (1 + exp(-z)). */
static double output_act(const o_cfg* c, double z)
{
    if (c->output == 1) return 1.0 / (1.0 + exp(-z));
    return exp(z < c->z_clamp ? z : c->z_clamp);
}

/* Cache value per RGB channel. */
static void cache_eval(const o_cfg* c, const double* params, const o_record* rec, const float w[3], double nval[3])
{
    double e[1024];
    double z[3];
    const double* hash = params + mlp_param_count(c);
    encode(c, hash, rec, w, e);
    mlp_forward(c, params, e, NULL, NULL, z);
    for (int k = 0; k < 3; k++) nval[k] = output_act(c, z[k]);
}

void orc_encode(const o_cfg* c, const double* params, const o_record* rec, const float w[3], double* e)
{
    encode(c, params + mlp_param_count(c), rec, w, e);
}

void orc_mlp(const o_cfg* c, const double* params, const double* e, double z[3])
{
    mlp_forward(c, params, e, NULL, NULL, z);
}

/* Bare cache queries: out[i] = n(record_i, dir_i). */
void orc_query(const o_cfg* c, const double* params, const o_record* recs, const float* dirs, uint64_t n,
               double* out)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < (int64_t)n; i++) cache_eval(c, params, &recs[i], dirs + 3 * i, out + 3 * i);
}

/* ------------------------------------------------------------------------ */
/* Path tracing: L_i(x, w) estimate along a direction (residual / training)  */
/* ------------------------------------------------------------------------ */

static const o_prim* scene_prims(const uint8_t* blob)
{
    return (const o_prim*)(blob + sizeof(o_header));
}

static void make_record(const o_prim* pr, uint32_t prim, const o_hit* h, const float d[3], o_record* rec)
{
    memset(rec, 0, sizeof(*rec));
    for (int k = 0; k < 3; k++) {
        rec->p[k] = h->p[k];
        rec->n[k] = h->n[k];
        rec->wo[k] = -d[k];
        rec->albedo[k] = pr->albedo[k];
    }
    rec->roughness = pr->roughness;
    rec->prim = prim;
    rec->flags = 1u | ((pr->flags & 3u) << 1);
}

/* ------------------------------------------------------------------------ */
/* Two-level estimation at later path vertices (estimator 2; paper:        */
/* "Biased and unbiased variants": NIRC at the first three vertices, and   */
/* the redistribution of neural samples between vertices)                   */
/* ------------------------------------------------------------------------ */

/* The residual path j of pixel pix reaches vertex x_k (k = 2, 3; x_1 is the
 * shading point) with throughput beta_k.  Its incident radiance there is
 * estimated by the same two levels (eq. L_mlmc applied recursively): the
 * path-traced continuation minus the cache's value for the continuation
 * direction w_k, plus N_k cache samples.  Along the path this adds
 *   beta_k C_k - beta_{k+1} n(x_k, w_k),  C_k = 1/N_k sum_i (f cos / p)_i n(x_k, w_i),
 * the second term only when the path continues (beta_{k+1} includes the
 * continuation weight and the Russian-roulette factor).  Both terms have
 * the same expectation, so the correction has mean zero for any cache. */
typedef struct {
    const o_cfg* c;
    const double* params;
    const o_frame* fd;
    uint32_t pix, j;
    double L[3];    /* sum of the corrections along the path */
    double Labs[3]; /* sum of their absolute values (the rounding scale of the sum) */
} o_mv;

static void cache_value(const o_cfg* c, const double* params, const o_frame* fd, const o_record* rec,
                        const float w[3], double nval[3]);

/* beta_k C_k at vertex k: N_k directions from purpose 10 + 16 k, counter (pix, j << 16 | i). */
static void mv_vertex(o_mv* mv, const o_record* rec, uint32_t k, const double beta[3])
{
    uint32_t nk = k == 2 ? mv->fd->n_cache2 : mv->fd->n_cache3;
    if (nk == 0) return;
    uint32_t k0 = (uint32_t)mv->fd->seed, k1 = mv->fd->frame;
    double C[3] = {0.0, 0.0, 0.0};
    for (uint32_t i = 0; i < nk; i++) {
        o_sample s;
        sample_bsdf(rec, k0, k1, mv->pix, (mv->j << 16) | i, PURPOSE_VCACHE + 16u * k, &s);
        if (!s.valid) continue;
        double nv[3];
        cache_value(mv->c, mv->params, mv->fd, rec, s.wi, nv);
        for (int q = 0; q < 3; q++) C[q] += s.w[q] * nv[q];
    }
    for (int q = 0; q < 3; q++) {
        mv->L[q] += beta[q] * C[q] / (double)nk;
        mv->Labs[q] += fabs(beta[q] * C[q] / (double)nk);
    }
}

/* - beta_{k+1} n(x_k, w_k) for the continuation direction (vertices with N_k = 0
 * use no cache at all). */
static void mv_continue(o_mv* mv, const o_record* rec, uint32_t k, const float wi[3], const double beta_next[3])
{
    if ((k == 2 ? mv->fd->n_cache2 : mv->fd->n_cache3) == 0) return;
    double nv[3];
    cache_value(mv->c, mv->params, mv->fd, rec, wi, nv);
    for (int q = 0; q < 3; q++) {
        mv->L[q] -= beta_next[q] * nv[q];
        mv->Labs[q] += fabs(beta_next[q] * nv[q]);
    }
}

/* Incident radiance along (o, d): emission at each vertex, BSDF-sampled
 * continuation, Russian roulette (continue with probability 0.9) before each
 * continuation, at most max_depth segments.  With mv, the two-level terms at
 * the path's vertices 2 and 3 (segments 1 and 2) go into mv->L. */
static void trace_path(const uint8_t* blob, const float o_in[3], const float d_in[3], uint32_t k0, uint32_t k1,
                       uint32_t c0, uint32_t c1, uint32_t max_depth, double L[3], uint64_t* sig, o_mv* mv)
{
    const o_header* hd = (const o_header*)blob;
    const o_prim* prims = scene_prims(blob);
    float o[3] = {o_in[0], o_in[1], o_in[2]};
    float d[3] = {d_in[0], d_in[1], d_in[2]};
    double beta[3] = {1.0, 1.0, 1.0};
    L[0] = L[1] = L[2] = 0.0;
    for (uint32_t seg = 1; seg <= max_depth; seg++) {
        float t;
        int prim = trace_nearest(prims, hd->n_prims, o, d, &t);
        *sig = sig_mix(*sig, prim < 0 ? 0xFFFFFFFFu : (uint32_t)prim);
        if (prim < 0) break;
        o_hit h;
        hit_info(&prims[prim], o, d, t, &h);
        double le[3];
        emitted(&prims[prim], h.front, le);
        for (int c = 0; c < 3; c++) L[c] += beta[c] * le[c];
        o_record rec;
        make_record(&prims[prim], (uint32_t)prim, &h, d, &rec);
        const int mv_here = mv && seg <= 2u;
        if (mv_here) mv_vertex(mv, &rec, seg + 1u, beta);
        if (seg == max_depth) break;
        uint32_t r[4];
        philox(k0, k1, c0, c1, 0u, PURPOSE_RR + 16u * seg, r);
        int cont = u01(r[0]) < RR_CONTINUE;
        *sig = sig_mix(*sig, (uint32_t)cont);
        if (!cont) break;
        for (int c = 0; c < 3; c++) beta[c] /= (double)RR_CONTINUE;
        o_sample s;
        sample_bsdf(&rec, k0, k1, c0, c1, PURPOSE_BOUNCE + 16u * seg, &s);
        *sig = sig_mix(*sig, sample_word(&s));
        if (!s.valid) break;
        for (int c = 0; c < 3; c++) beta[c] *= s.w[c];
        if (mv_here) mv_continue(mv, &rec, seg + 1u, s.wi, beta);
        for (int k = 0; k < 3; k++) {
            o[k] = h.p[k];
            d[k] = s.wi[k];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Next-event estimation with multiple importance sampling (light mode 1)   */
/* ------------------------------------------------------------------------ */

#define MAX_LIGHTS 1024

typedef struct {
    uint32_t n;
    uint32_t idx[MAX_LIGHTS]; /* emitting rectangles in primitive order */
} o_lights;

static int is_rect_emitter(const o_prim* p)
{
    return p->kind == KIND_RECT && (p->emission[0] > 0.0f || p->emission[1] > 0.0f || p->emission[2] > 0.0f);
}

static void collect_lights(const uint8_t* blob, o_lights* L)
{
    const o_header* hd = (const o_header*)blob;
    const o_prim* prims = scene_prims(blob);
    L->n = 0;
    for (uint32_t i = 0; i < hd->n_prims && L->n < MAX_LIGHTS; i++)
        if (is_rect_emitter(&prims[i])) L->idx[L->n++] = i;
}

static double rect_area(const o_prim* p)
{
    double u[3] = {p->u[0], p->u[1], p->u[2]}, v[3] = {p->v[0], p->v[1], p->v[2]};
    double c[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
    return sqrt(dot3d(c, c));
}

/* f_r cos(theta_i) and the BSDF sampling density p(wi) (solid angle) of the
 * material at rec for an arbitrary direction wi; both 0 below the surface. */
static void bsdf_eval(const o_record* rec, const float wif[3], double fcos[3], double* pdf)
{
    uint32_t mat = (rec->flags >> 1) & 3u;
    double n[3] = {rec->n[0], rec->n[1], rec->n[2]};
    double wi[3] = {wif[0], wif[1], wif[2]};
    double ci = dot3d(n, wi);
    fcos[0] = fcos[1] = fcos[2] = 0.0;
    *pdf = 0.0;
    if (mat == MAT_BLACK || !(ci > 0.0)) return;
    if (mat == MAT_LAMBERT) {
        for (int c = 0; c < 3; c++) fcos[c] = (double)rec->albedo[c] / O_PI * ci;
        *pdf = ci / O_PI;
        return;
    }
    double wo[3] = {rec->wo[0], rec->wo[1], rec->wo[2]};
    double alpha = (double)(rec->roughness * rec->roughness);
    double a2 = alpha * alpha;
    double co = dot3d(n, wo);
    double h[3] = {wo[0] + wi[0], wo[1] + wi[1], wo[2] + wi[2]};
    double hl = sqrt(dot3d(h, h));
    for (int k = 0; k < 3; k++) h[k] /= hl;
    double oh = dot3d(wo, h);
    if (oh < 0.0) oh = 0.0;
    if (oh > 1.0) oh = 1.0;
    double dd = ggx_dd(n, h, a2);
    double D = a2 / (O_PI * dd * dd);
    double lam_o = sqrt(a2 + (1.0 - a2) * co * co);
    double lam_i = sqrt(a2 + (1.0 - a2) * ci * ci);
    double G2 = 2.0 * ci * co / (co * lam_i + ci * lam_o);
    double G1o = 2.0 * co / (co + lam_o);
    double F = F0_SPEC + (1.0 - F0_SPEC) * pow(1.0 - oh, 5.0);
    double fs = F * D * G2 / (4.0 * ci * co);
    for (int c = 0; c < 3; c++) fcos[c] = ((double)rec->albedo[c] / O_PI + fs) * ci;
    *pdf = 0.5 * ci / O_PI + 0.5 * G1o * D / (4.0 * co);
}

/* Solid-angle density of sampling direction d toward a point at distance t
 * on emitting rectangle e by the light technique (uniform emitter, uniform
 * point). */
static double light_pdf(const o_prim* e, const float d[3], double t, uint32_t n_lights)
{
    double cl = fabs((double)e->n[0] * d[0] + (double)e->n[1] * d[1] + (double)e->n[2] * d[2]);
    return t * t / (cl * rect_area(e) * (double)n_lights);
}

/* Power-heuristic weight of technique a (n_a samples, density pa) against b. */
static double power_weight(double na_pa, double nb_pb)
{
    double a = na_pa * na_pa, b = nb_pb * nb_pb;
    return a + b > 0.0 ? a / (a + b) : 0.0;
}

/* One light sample at shading record rec: emitter k uniform among the
 * rectangles (word 0), point a + u1 U + u2 V (words 1, 2), shadow ray,
 * contribution f cos L_e cos_l / (dist^2 pdf_area), weighted against n_b BSDF
 * samples by the power heuristic.  Adds into out; returns the decision word
 * (emitter | geometry ok << 16 | visible << 17) for the signature. */
static uint32_t nee_sample(const uint8_t* blob, const o_lights* lights, const o_record* rec, uint32_t n_b,
                           uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c3, double out[3])
{
    const o_header* hd = (const o_header*)blob;
    const o_prim* prims = scene_prims(blob);
    if (lights->n == 0 || ((rec->flags >> 1) & 3u) == MAT_BLACK) return 0;
    uint32_t r[4];
    philox(k0, k1, c0, c1, 0u, c3, r);
    uint32_t e = (uint32_t)(((uint64_t)r[0] * lights->n) >> 32);
    uint32_t li = lights->idx[e];
    const o_prim* L = &prims[li];
    float u1 = u01(r[1]), u2 = u01(r[2]);
    float pt[3], v[3], w[3];
    for (int k = 0; k < 3; k++) {
        pt[k] = (L->a[k] + u1 * L->u[k]) + u2 * L->v[k];
        v[k] = pt[k] - rec->p[k];
    }
    float dist2 = dot3f(v, v);
    float dist = sqrtf(dist2);
    w[0] = v[0];
    w[1] = v[1];
    w[2] = v[2];
    normalize3f(w);
    float cx = dot3f(rec->n, w);
    float cl = -dot3f(L->n, w);
    int ok = cx > 0.0f && (cl > 0.0f || ((L->flags & EMIT_TWO_SIDED) && cl < 0.0f));
    uint32_t word = e | ((uint32_t)ok << 16);
    if (!ok) return word;
    float t;
    int hit = trace_nearest(prims, hd->n_prims, rec->p, w, &t);
    int visible = hit == (int)li && fabsf(t - dist) <= 1e-3f * dist;
    word |= (uint32_t)visible << 17;
    if (!visible) return word;
    double fcos[3], pb;
    bsdf_eval(rec, w, fcos, &pb);
    double pl = light_pdf(L, w, (double)dist, lights->n);
    double wl = power_weight(pl, (double)n_b * pb);
    for (int c = 0; c < 3; c++) out[c] += fcos[c] * (double)L->emission[c] * wl / pl;
    return word;
}

/* L_ind(x, d): the path from o along d, NEE at every vertex (MIS against the
 * continuation, except at the last vertex, which has none), emission found
 * by a continuation weighted by the power heuristic.  The emission of the
 * first hit is not part of L_ind; it is returned in first_emit, weighted for
 * the shading point's MIS (n_b0 BSDF samples of density pb0 there). */
static void trace_path_nee(const uint8_t* blob, const o_lights* lights, const float o_in[3], const float d_in[3],
                           uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t max_depth, uint32_t n_b0,
                           double pb0, double L[3], double first_emit[3], uint64_t* sig, o_mv* mv)
{
    const o_header* hd = (const o_header*)blob;
    const o_prim* prims = scene_prims(blob);
    float o[3] = {o_in[0], o_in[1], o_in[2]};
    float d[3] = {d_in[0], d_in[1], d_in[2]};
    double beta[3] = {1.0, 1.0, 1.0};
    double pb_prev = pb0;
    L[0] = L[1] = L[2] = 0.0;
    first_emit[0] = first_emit[1] = first_emit[2] = 0.0;
    for (uint32_t seg = 1; seg <= max_depth; seg++) {
        float t;
        int prim = trace_nearest(prims, hd->n_prims, o, d, &t);
        *sig = sig_mix(*sig, prim < 0 ? 0xFFFFFFFFu : (uint32_t)prim);
        if (prim < 0) break;
        o_hit h;
        hit_info(&prims[prim], o, d, t, &h);
        double le[3];
        emitted(&prims[prim], h.front, le);
        if (le[0] > 0.0 || le[1] > 0.0 || le[2] > 0.0) {
            uint32_t nb = seg == 1 ? n_b0 : 1u;
            double wb = 1.0;
            if (is_rect_emitter(&prims[prim]) && lights->n)
                wb = power_weight((double)nb * pb_prev, light_pdf(&prims[prim], d, (double)t, lights->n));
            if (seg == 1) {
                for (int c = 0; c < 3; c++) first_emit[c] = le[c] * wb;
            } else {
                for (int c = 0; c < 3; c++) L[c] += beta[c] * le[c] * wb;
            }
        }
        o_record rec;
        make_record(&prims[prim], (uint32_t)prim, &h, d, &rec);
        double dl[3] = {0.0, 0.0, 0.0};
        *sig = sig_mix(*sig, nee_sample(blob, lights, &rec, seg < max_depth ? 1u : 0u, k0, k1, c0, c1,
                                        PURPOSE_LIGHT + 16u * seg, dl));
        for (int c = 0; c < 3; c++) L[c] += beta[c] * dl[c];
        const int mv_here = mv && seg <= 2u;
        if (mv_here) mv_vertex(mv, &rec, seg + 1u, beta);
        if (seg == max_depth) break;
        uint32_t r[4];
        philox(k0, k1, c0, c1, 0u, PURPOSE_RR + 16u * seg, r);
        int cont = u01(r[0]) < RR_CONTINUE;
        *sig = sig_mix(*sig, (uint32_t)cont);
        if (!cont) break;
        for (int c = 0; c < 3; c++) beta[c] /= (double)RR_CONTINUE;
        o_sample s;
        sample_bsdf(&rec, k0, k1, c0, c1, PURPOSE_BOUNCE + 16u * seg, &s);
        *sig = sig_mix(*sig, sample_word(&s));
        if (!s.valid) break;
        for (int c = 0; c < 3; c++) beta[c] *= s.w[c];
        if (mv_here) mv_continue(mv, &rec, seg + 1u, s.wi, beta);
        double fc[3];
        bsdf_eval(&rec, s.wi, fc, &pb_prev);
        for (int k = 0; k < 3; k++) {
            o[k] = h.p[k];
            d[k] = s.wi[k];
        }
    }
}

/* Camera ray through pixel (px, py) with jitter (jx, jy). */
static void camera_ray(const o_header* hd, uint32_t W, uint32_t H, uint32_t px, uint32_t py, float jx, float jy,
                       float o[3], float d[3])
{
    float s = ((float)px + jx) / (float)W;
    float t = ((float)py + jy) / (float)H;
    for (int k = 0; k < 3; k++) {
        o[k] = hd->origin[k];
        d[k] = ((hd->top_left[k] + s * hd->horizontal[k]) + t * hd->vertical[k]) - hd->origin[k];
    }
    normalize3f(d);
}

/* ------------------------------------------------------------------------ */
/* Environment map (light mode 2): a cube map stored after the primitives   */
/* ------------------------------------------------------------------------ */

/* Face size S of the scene's cube map (header word reserved[0]; 0: none);
 * its 6 S S texels (RGB + pad, float) follow the primitives, face-major,
 * then row, then column. */
static uint32_t env_size(const uint8_t* blob)
{
    return ((const o_header*)blob)->reserved[0];
}

/* Texel of direction d: the major axis picks the face (ties: x before y
 * before z; face 0 +x, 1 -x, 2 +y, 3 -y, 4 +z, 5 -z), the other two
 * coordinates in axis order (a, b) over |major| map [-1, 1] to [0, S)
 * (column from a, row from b, clamped to S - 1).  Strict binary32: it picks
 * an integer. */
static uint32_t env_texel(uint32_t S, const float d[3])
{
    float ax = fabsf(d[0]), ay = fabsf(d[1]), az = fabsf(d[2]);
    uint32_t face;
    float m, a, b;
    if (ax >= ay && ax >= az) {
        face = d[0] >= 0.0f ? 0u : 1u;
        m = ax;
        a = d[1];
        b = d[2];
    } else if (ay >= az) {
        face = d[1] >= 0.0f ? 2u : 3u;
        m = ay;
        a = d[0];
        b = d[2];
    } else {
        face = d[2] >= 0.0f ? 4u : 5u;
        m = az;
        a = d[0];
        b = d[1];
    }
    float u = (a / m + 1.0f) * 0.5f, v = (b / m + 1.0f) * 0.5f;
    uint32_t i = (uint32_t)floorf(u * (float)S), j = (uint32_t)floorf(v * (float)S);
    if (i >= S) i = S - 1;
    if (j >= S) j = S - 1;
    return face * S * S + j * S + i;
}

/* L_env(d): the texel's radiance (nearest texel), 0 without a map. */
static void env_radiance(const uint8_t* blob, const float d[3], double L[3])
{
    uint32_t S = env_size(blob);
    L[0] = L[1] = L[2] = 0.0;
    if (!S) return;
    const o_header* hd = (const o_header*)blob;
    const float* tex = (const float*)(blob + sizeof(o_header) + (size_t)hd->n_prims * sizeof(o_prim));
    uint32_t t = env_texel(S, d);
    for (int k = 0; k < 3; k++) L[k] = (double)tex[4 * (size_t)t + k];
}

/* A visibility cache's value times the environment's radiance. */
static void env_factor(const uint8_t* blob, const float d[3], double nv[3])
{
    double L[3];
    env_radiance(blob, d, L);
    for (int k = 0; k < 3; k++) nv[k] *= L[k];
}

uint32_t orc_env_texel(uint32_t S, const float d[3])
{
    return env_texel(S, d);
}

/* ------------------------------------------------------------------------ */
/* Two-level estimator per pixel:                                           */
/*   L_o = L_e + L_c + L_r                                (eq. L_mlmc)      */
/*   L_c = 1/N_c sum_i n(x, w_i) f_r cos / p              (eq. L_c)         */
/*   L_r = 1/N_r sum_j (L_i(x, w_j) - n(x, w_j)) f_r cos / p   (eq. L_r)    */
/* with independent BSDF-sampled direction sets for the two levels.         */
/* ------------------------------------------------------------------------ */

static void cache_value(const o_cfg* c, const double* params, const o_frame* fd, const o_record* rec,
                        const float w[3], double nval[3])
{
    if (fd->cache_mode == 1) {
        nval[0] = nval[1] = nval[2] = 0.0;
    } else if (fd->cache_mode == 2) {
        for (int k = 0; k < 3; k++) nval[k] = fd->cache_const[k];
    } else {
        cache_eval(c, params, rec, w, nval);
    }
}

static void estimate_pixel(const o_cfg* c, const double* params, const uint8_t* blob, const o_frame* fd,
                           const o_lights* lights, uint32_t pix, double out[3], double lc_out[3], double lr_out[3],
                           uint64_t sig[2], uint32_t* count, double* row_n, double lr_abs[3])
{
    /* lr_abs (optional): the sum of the absolute values of the terms that
     * make up L_r, the scale of its rounding error (the terms cancel) */
    double Labs[3] = {0.0, 0.0, 0.0};
    /* light mode 2 with a visibility cache: n = V(x, w) L_env(w) */
    const int env = fd->light_mode == 2 && c->output == 1;
    /* row_n (optional): cache value of each of the N + M rows, 0 for rows
     * whose sample is invalid or whose pixel has no camera hit */
    if (row_n) memset(row_n, 0, 3 * sizeof(double) * (fd->n_cache + fd->n_resid));
    const o_header* hd = (const o_header*)blob;
    const o_prim* prims = scene_prims(blob);
    uint32_t k0 = (uint32_t)fd->seed, k1 = fd->frame;
    uint32_t px = pix % fd->width, py = pix / fd->width;
    uint64_t sp = SIG_INIT, sc = SIG_INIT;
    uint32_t active = 0;
    double Le[3] = {0, 0, 0}, Lc[3] = {0, 0, 0}, Lr[3] = {0, 0, 0};

    uint32_t r[4];
    philox(k0, k1, pix, 0u, 0u, PURPOSE_CAMERA, r);
    float o[3], d[3];
    camera_ray(hd, fd->width, fd->height, px, py, u01(r[0]), u01(r[1]), o, d);
    float t;
    int prim = trace_nearest(prims, hd->n_prims, o, d, &t);
    sp = sig_mix(sp, prim < 0 ? 0xFFFFFFFFu : (uint32_t)prim);
    if (prim >= 0) {
        o_hit h;
        hit_info(&prims[prim], o, d, t, &h);
        emitted(&prims[prim], h.front, Le);
        o_record rec;
        make_record(&prims[prim], (uint32_t)prim, &h, d, &rec);
        if (lights) {
            /* direct light at x: one light sample against the M residual directions */
            double dl[3] = {0.0, 0.0, 0.0};
            sp = sig_mix(sp, nee_sample(blob, lights, &rec, fd->n_resid, k0, k1, pix, 0u, PURPOSE_LIGHT, dl));
            for (int k = 0; k < 3; k++) Le[k] += dl[k];
        }

        for (uint32_t i = 0; i < fd->n_cache; i++) {
            o_sample s;
            sample_bsdf(&rec, k0, k1, pix, i, PURPOSE_CACHE_DIR, &s);
            sc = sig_mix(sc, sample_word(&s));
            if (!s.valid) continue;
            double nv[3];
            cache_value(c, params, fd, &rec, s.wi, nv);
            if (env) env_factor(blob, s.wi, nv);
            for (int k = 0; k < 3; k++) Lc[k] += s.w[k] * nv[k];
            if (row_n)
                for (int k = 0; k < 3; k++) row_n[3 * i + k] = nv[k];
            active++;
        }
        if (fd->n_cache) for (int k = 0; k < 3; k++) Lc[k] /= (double)fd->n_cache;

        for (uint32_t j = 0; j < fd->n_resid; j++) {
            o_sample s;
            sample_bsdf(&rec, k0, k1, pix, j, PURPOSE_RESID_DIR, &s);
            sp = sig_mix(sp, sample_word(&s));
            if (!s.valid) continue;
            double Li[3], nv[3];
            o_mv mv = {c, params, fd, pix, j, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
            o_mv* mvp = fd->estimator == 2 ? &mv : NULL;
            if (fd->light_mode == 2) {
                /* direct environment light: V(x, w_j) L_env(w_j), one ray */
                float tv;
                int q = trace_nearest(prims, hd->n_prims, rec.p, s.wi, &tv);
                sp = sig_mix(sp, q < 0 ? 0xFFFFFFFFu : (uint32_t)q);
                if (q < 0) {
                    env_radiance(blob, s.wi, Li);
                } else {
                    Li[0] = Li[1] = Li[2] = 0.0;
                }
            } else if (lights) {
                double fc[3], pb, e1[3];
                bsdf_eval(&rec, s.wi, fc, &pb);
                trace_path_nee(blob, lights, rec.p, s.wi, k0, k1, pix, j, fd->max_depth, fd->n_resid, pb, Li, e1,
                               &sp, mvp);
                for (int k = 0; k < 3; k++) Le[k] += s.w[k] * e1[k] / (double)fd->n_resid;
            } else {
                trace_path(blob, rec.p, s.wi, k0, k1, pix, j, fd->max_depth, Li, &sp, mvp);
            }
            cache_value(c, params, fd, &rec, s.wi, nv);
            if (env) env_factor(blob, s.wi, nv);
            /* with N = 0 there is no cache level, and nothing is subtracted */
            const double use = fd->n_cache ? 1.0 : 0.0;
            for (int k = 0; k < 3; k++) {
                Lr[k] += s.w[k] * (Li[k] - use * nv[k] + mv.L[k]);
                Labs[k] += fabs(s.w[k]) * (fabs(Li[k]) + use * fabs(nv[k]) + mv.Labs[k]);
            }
            if (row_n)
                for (int k = 0; k < 3; k++) row_n[3 * (fd->n_cache + j) + k] = nv[k];
            active++;
        }
        if (fd->n_resid)
            for (int k = 0; k < 3; k++) {
                Lr[k] /= (double)fd->n_resid;
                Labs[k] /= (double)fd->n_resid;
            }
    }
    if (lr_abs)
        for (int k = 0; k < 3; k++) lr_abs[k] = Labs[k];
    for (int k = 0; k < 3; k++) {
        out[k] = Le[k] + Lc[k] + Lr[k];
        if (lc_out) lc_out[k] = Lc[k];
        if (lr_out) lr_out[k] = Lr[k];
    }
    if (sig) {
        sig[0] = sp;
        sig[1] = sc;
    }
    if (count) *count = active;
}

/* ------------------------------------------------------------------------ */
/* Path termination (paper: section "Path Termination Heuristics")          */
/* ------------------------------------------------------------------------ */

/* Density of the BSDF sampler at wi (the p of the termination tests) in
 * strict binary32, fixed operation order: it decides whether a path goes on,
 * so both implementations compute it identically.  Lambertian: cos/pi;
 * Lambertian + GGX: the one-sample mixture 1/2 cos/pi + 1/2 G1(wo) D / (4
 * cos_o), D = a2 / (pi dd^2), dd = |n x h|^2 + a2 (n.h)^2, a = roughness^2. */
static float sampler_pdf32(const o_record* rec, const float wi[3])
{
    const float inv_pi = (float)(1.0 / O_PI);
    uint32_t mat = (rec->flags >> 1) & 3u;
    float ci = dot3f(rec->n, wi);
    if (mat == MAT_BLACK || !(ci > 0.0f)) return 0.0f;
    if (mat == MAT_LAMBERT) return ci * inv_pi;
    const float* n = rec->n;
    float co = dot3f(n, rec->wo);
    float h[3] = {rec->wo[0] + wi[0], rec->wo[1] + wi[1], rec->wo[2] + wi[2]};
    normalize3f(h);
    float a = rec->roughness * rec->roughness;
    float a2 = a * a;
    float cnh = dot3f(n, h);
    float cx[3] = {n[1] * h[2] - n[2] * h[1], n[2] * h[0] - n[0] * h[2], n[0] * h[1] - n[1] * h[0]};
    float dd = dot3f(cx, cx) + a2 * (cnh * cnh);
    float D = a2 / (((float)O_PI * dd) * dd);
    float lam_o = sqrtf(a2 + (1.0f - a2) * (co * co));
    float g1 = (2.0f * co) / (co + lam_o);
    return 0.5f * (ci * inv_pi) + 0.5f * ((g1 * D) / (4.0f * co));
}

/* Balanced Termination Heuristic: continuation probability
 * P_s = p / (p + N_c / pi) of a path whose sampled direction has density p,
 * N_c neural samples (binary32). */
static float bth_continue_prob(float p, uint32_t n_c)
{
    return p / (p + (float)n_c * (float)(1.0 / O_PI));
}

/* Spread-angle footprint term of one segment of length t arriving at a
 * vertex at cosine cos_in, sampled with density p at the previous vertex
 * (NRC's heuristic, which the paper uses for vertices after the first):
 *   a(x_1 .. x_n) = (sum_{i=2..n} sqrt(|x_{i-1} - x_i|^2 / (p cos_i)))^2,
 *   a_0 = |x_0 - x_1|^2 / (4 pi cos_1),  stop when a > c a_0, c = 0.01. */
static float spread_term(float t, float p, float cos_in)
{
    return sqrtf((t * t) / (p * cos_in));
}

/* The camera path of the biased estimator (paper: "Biased and unbiased
 * variants" and the termination criteria of section "Path Termination
 * Heuristics"): from vertex x_i the path continues with the BSDF-sampled
 * direction w_i while xi_i <= P_s(w_i) and, for i > 1, the footprint
 * a(x_1..x_i) stays within c a_0; it stops there otherwise, or at vertex
 * max_depth.  Emission found along the path is added to le with the path
 * throughput; in light mode 1 every vertex takes a light sample (NEE) and
 * w_i is the BSDF technique of the power heuristic (one sample), traced at
 * the stopping vertex too, for its emission only.  No Russian roulette: the
 * termination tests and the depth cap end the path.  Returns the index of
 * the stopping vertex (its record in term, the throughput up to it in beta)
 * or 0 when the path left the scene first. */
static uint32_t bth_path(const uint8_t* blob, const o_frame* fd, const o_lights* lights, uint32_t pix,
                         o_record* term, double beta[3], double Le[3], uint64_t* sig)
{
    const o_header* hd = (const o_header*)blob;
    const o_prim* prims = scene_prims(blob);
    uint32_t k0 = (uint32_t)fd->seed, k1 = fd->frame;
    uint32_t px = pix % fd->width, py = pix / fd->width;
    uint64_t sp = SIG_INIT;
    uint32_t stop_at = 0;
    for (int k = 0; k < 3; k++) {
        Le[k] = 0.0;
        beta[k] = 1.0;
    }
    memset(term, 0, sizeof(*term));

    uint32_t r[4];
    philox(k0, k1, pix, 0u, 0u, PURPOSE_CAMERA, r);
    float o[3], d[3];
    camera_ray(hd, fd->width, fd->height, px, py, u01(r[0]), u01(r[1]), o, d);
    float t;
    int prim = trace_nearest(prims, hd->n_prims, o, d, &t);
    sp = sig_mix(sp, prim < 0 ? 0xFFFFFFFFu : (uint32_t)prim);
    if (prim >= 0) {
        o_hit h;
        hit_info(&prims[prim], o, d, t, &h);
        emitted(&prims[prim], h.front, Le);
        const float c_a0 = 0.01f * ((t * t) / ((4.0f * (float)O_PI) * fabsf(dot3f(h.n, d))));
        float spread = 0.0f;
        for (uint32_t i = 1;; i++) {
            o_record rec;
            make_record(&prims[prim], (uint32_t)prim, &h, d, &rec);
            if (lights) {
                double dl[3] = {0.0, 0.0, 0.0};
                sp = sig_mix(sp, nee_sample(blob, lights, &rec, 1u, k0, k1, pix, 0u, PURPOSE_LIGHT + 16u * i, dl));
                for (int k = 0; k < 3; k++) Le[k] += beta[k] * dl[k];
            }
            o_sample s;
            sample_bsdf(&rec, k0, k1, pix, 0u, PURPOSE_BTH_DIR + 16u * i, &s);
            sp = sig_mix(sp, sample_word(&s));
            float p = s.valid ? sampler_pdf32(&rec, s.wi) : 0.0f;
            philox(k0, k1, pix, 0u, 0u, PURPOSE_BTH_XI + 16u * i, r);
            uint32_t stop = (uint32_t)(u01(r[0]) > bth_continue_prob(p, fd->n_cache));
            if (i > 1 && spread * spread > c_a0) stop |= 2u;
            if (i == fd->max_depth) stop |= 4u;
            sp = sig_mix(sp, stop);
            if (stop) {
                *term = rec;
                stop_at = i;
                if (lights && s.valid) {
                    /* the BSDF technique of the direct light at the stopping vertex */
                    int q = trace_nearest(prims, hd->n_prims, rec.p, s.wi, &t);
                    sp = sig_mix(sp, q < 0 ? 0xFFFFFFFFu : (uint32_t)q);
                    if (q >= 0) {
                        o_hit hq;
                        hit_info(&prims[q], rec.p, s.wi, t, &hq);
                        double le[3];
                        emitted(&prims[q], hq.front, le);
                        double wb = 1.0;
                        if (is_rect_emitter(&prims[q]) && lights->n) {
                            double fc[3], pb;
                            bsdf_eval(&rec, s.wi, fc, &pb);
                            wb = power_weight(pb, light_pdf(&prims[q], s.wi, (double)t, lights->n));
                        }
                        for (int k = 0; k < 3; k++) Le[k] += beta[k] * s.w[k] * le[k] * wb;
                    }
                }
                break;
            }
            /* continue along w_i */
            double pb = 0.0;
            if (lights) {
                double fc[3];
                bsdf_eval(&rec, s.wi, fc, &pb);
            }
            for (int k = 0; k < 3; k++) beta[k] *= s.w[k];
            for (int k = 0; k < 3; k++) {
                o[k] = rec.p[k];
                d[k] = s.wi[k];
            }
            prim = trace_nearest(prims, hd->n_prims, o, d, &t);
            sp = sig_mix(sp, prim < 0 ? 0xFFFFFFFFu : (uint32_t)prim);
            if (prim < 0) break;
            hit_info(&prims[prim], o, d, t, &h);
            double le[3];
            emitted(&prims[prim], h.front, le);
            double wb = 1.0;
            if (lights && is_rect_emitter(&prims[prim]) && lights->n)
                wb = power_weight(pb, light_pdf(&prims[prim], d, (double)t, lights->n));
            for (int k = 0; k < 3; k++) Le[k] += beta[k] * le[k] * wb;
            spread = spread + spread_term(t, p, fabsf(dot3f(h.n, d)));
        }
    }
    *sig = sp;
    return stop_at;
}

/* The biased estimator per pixel: the camera path above, then N_c cache
 * samples at its stopping vertex (eq. L_c) times the path throughput; no
 * residual level. */
static void estimate_pixel_bth(const o_cfg* c, const double* params, const uint8_t* blob, const o_frame* fd,
                               const o_lights* lights, uint32_t pix, double out[3], double lc_out[3],
                               double lr_out[3], uint64_t sig[2], uint32_t* count, double* row_n, double lr_abs[3])
{
    if (lr_abs) lr_abs[0] = lr_abs[1] = lr_abs[2] = 0.0;
    if (row_n) memset(row_n, 0, 3 * sizeof(double) * fd->n_cache);
    uint32_t k0 = (uint32_t)fd->seed, k1 = fd->frame;
    uint64_t sp, sc = SIG_INIT;
    uint32_t active = 0;
    double Le[3], beta[3], Lc[3] = {0, 0, 0};
    o_record term;
    uint32_t at = bth_path(blob, fd, lights, pix, &term, beta, Le, &sp);
    if (at) {
        for (uint32_t i = 0; i < fd->n_cache; i++) {
            o_sample s;
            sample_bsdf(&term, k0, k1, pix, i, PURPOSE_CACHE_DIR, &s);
            sc = sig_mix(sc, sample_word(&s));
            if (!s.valid) continue;
            double nv[3];
            cache_value(c, params, fd, &term, s.wi, nv);
            for (int k = 0; k < 3; k++) Lc[k] += s.w[k] * nv[k];
            if (row_n)
                for (int k = 0; k < 3; k++) row_n[3 * i + k] = nv[k];
            active++;
        }
        if (fd->n_cache)
            for (int k = 0; k < 3; k++) Lc[k] *= beta[k] / (double)fd->n_cache;
    }
    for (int k = 0; k < 3; k++) {
        out[k] = Le[k] + Lc[k];
        if (lc_out) lc_out[k] = Lc[k];
        if (lr_out) lr_out[k] = 0.0;
    }
    if (sig) {
        sig[0] = sp;
        sig[1] = sc;
    }
    if (count) *count = active;
}

/* The camera path of the biased estimator for one pixel (test access):
 * returns the stopping vertex (0: none) with its record, the throughput up
 * to it and the radiance collected on the way. */
uint32_t orc_bth_path(const uint8_t* blob, const o_frame* fd, uint32_t pix, o_record* term, double beta[3],
                      double le[3], uint64_t* sig)
{
    o_lights* lights = NULL;
    if (fd->light_mode == 1) {
        lights = (o_lights*)malloc(sizeof(o_lights));
        collect_lights(blob, lights);
    }
    uint32_t at = bth_path(blob, fd, lights, pix, term, beta, le, sig);
    free(lights);
    return at;
}

float orc_sampler_pdf32(const o_record* rec, const float wi[3])
{
    return sampler_pdf32(rec, wi);
}

/* Estimate the listed pixels (all W*H when pixels == NULL).  Outputs are
 * indexed by position in the list; optional outputs may be NULL. */
void orc_estimate_pixels(const o_cfg* c, const double* params, const uint8_t* blob, const o_frame* fd,
                         const uint32_t* pixels, uint64_t n, double* out, double* lc, double* lr, uint64_t* sig,
                         uint32_t* count, double* row_n, double* lr_abs)
{
    const uint64_t S = (uint64_t)fd->n_cache + fd->n_resid;
    o_lights* lights = NULL;
    if (fd->light_mode == 1) {
        lights = (o_lights*)malloc(sizeof(o_lights));
        collect_lights(blob, lights);
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < (int64_t)n; i++) {
        uint32_t pix = pixels ? pixels[i] : (uint32_t)i;
        if (fd->estimator == 1)
            estimate_pixel_bth(c, params, blob, fd, lights, pix, out + 3 * i, lc ? lc + 3 * i : NULL,
                               lr ? lr + 3 * i : NULL, sig ? sig + 2 * i : NULL, count ? count + i : NULL,
                               row_n ? row_n + 3 * S * i : NULL, lr_abs ? lr_abs + 3 * i : NULL);
        else
            estimate_pixel(c, params, blob, fd, lights, pix, out + 3 * i, lc ? lc + 3 * i : NULL,
                           lr ? lr + 3 * i : NULL, sig ? sig + 2 * i : NULL, count ? count + i : NULL,
                           row_n ? row_n + 3 * S * i : NULL, lr_abs ? lr_abs + 3 * i : NULL);
    }
    free(lights);
}

/* ------------------------------------------------------------------------ */
/* Training records: a separate path-tracing pass (one record per path,     */
/* at its first vertex; target = path-traced incident radiance)              */
/* ------------------------------------------------------------------------ */

void orc_gen_train(const uint8_t* blob, uint32_t W, uint32_t H, uint64_t T, uint32_t frame, uint64_t seed,
                   uint32_t max_depth, uint32_t light_mode, uint32_t visibility, o_record* recs, float* dirs,
                   double* targets, uint64_t* sig)
{
    /* light mode 2: the target is the direct environment light V L_env
     * along the sampled direction, or V alone for a visibility cache */
    const o_header* hd = (const o_header*)blob;
    const o_prim* prims = scene_prims(blob);
    uint32_t k0 = (uint32_t)seed, k1 = frame ^ 0x80000000u;
    uint64_t P = (uint64_t)W * H;
    o_lights* lights = NULL;
    if (light_mode == 1) {
        lights = (o_lights*)malloc(sizeof(o_lights));
        collect_lights(blob, lights);
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t ti = 0; ti < (int64_t)T; ti++) {
        uint32_t tr = (uint32_t)ti;
        uint32_t r[4];
        philox(k0, k1, tr, 0u, 0u, PURPOSE_TRAIN_PICK, r);
        uint32_t pix = (uint32_t)(((uint64_t)r[0] * P) >> 32);
        uint64_t sg = SIG_INIT;
        sg = sig_mix(sg, pix);
        float o[3], d[3];
        camera_ray(hd, W, H, pix % W, pix / W, u01(r[1]), u01(r[2]), o, d);
        float t;
        int prim = trace_nearest(prims, hd->n_prims, o, d, &t);
        sg = sig_mix(sg, prim < 0 ? 0xFFFFFFFFu : (uint32_t)prim);
        o_record rec;
        memset(&rec, 0, sizeof(rec));
        float* dir = dirs + 3 * ti;
        double* tg = targets + 3 * ti;
        dir[0] = dir[1] = dir[2] = 0.0f;
        tg[0] = tg[1] = tg[2] = 0.0;
        if (prim >= 0) {
            o_hit h;
            hit_info(&prims[prim], o, d, t, &h);
            make_record(&prims[prim], (uint32_t)prim, &h, d, &rec);
            o_sample s;
            sample_bsdf(&rec, k0, k1, tr, 0u, PURPOSE_RESID_DIR, &s);
            sg = sig_mix(sg, sample_word(&s));
            if (s.valid) {
                if (light_mode == 2) {
                    float tv;
                    int q = trace_nearest(prims, hd->n_prims, rec.p, s.wi, &tv);
                    sg = sig_mix(sg, q < 0 ? 0xFFFFFFFFu : (uint32_t)q);
                    if (q < 0) {
                        if (visibility) {
                            tg[0] = tg[1] = tg[2] = 1.0;
                        } else {
                            env_radiance(blob, s.wi, tg);
                        }
                    }
                } else if (lights) {
                    /* target = L_ind: the first hit's emission is direct light */
                    double e1[3];
                    trace_path_nee(blob, lights, rec.p, s.wi, k0, k1, tr, 0u, max_depth, 0u, 0.0, tg, e1, &sg, NULL);
                } else {
                    trace_path(blob, rec.p, s.wi, k0, k1, tr, 0u, max_depth, tg, &sg, NULL);
                }
                for (int k = 0; k < 3; k++) dir[k] = s.wi[k];
            } else {
                rec.flags &= ~1u; /* no usable direction: excluded from the loss */
            }
        }
        recs[ti] = rec;
        if (sig) sig[ti] = sg;
    }
    free(lights);
}

/* ------------------------------------------------------------------------ */
/* Relative L2 loss (eq. 12) with p_r = 1, and its exact gradient           */
/*   L = 1/(3T) sum_t sum_ch valid_t (f - n)^2 / (sg(n)^2 + eps)             */
/* ------------------------------------------------------------------------ */

/* Returns the loss; adds dL/dparams into grad (length orc_param_count).
 * The stop-gradient denominator sg(n)^2 + eps is taken from the current
 * network unless den_fixed (T x 3) is given, in which case it is used for
 * both the loss and the gradient: the loss is then a plain function of the
 * parameters whose derivative at the point where den_fixed was taken is the
 * training gradient (used by the finite-difference pin). */
/* Shared core of the training loss gradient and of the query gradient.
 * With gout == NULL it is the loss above (valid records only); with gout
 * (T x 3) given it returns sum_t sum_ch gout * n over every record and adds
 * the gradient of that sum, i.e. the vector-Jacobian product of eq. 11's
 * cache with the upstream gradient gout. */
static double loss_grad_core(const o_cfg* c, const double* params, const o_record* recs, const float* dirs,
                             const double* targets, const double* gout, uint64_t T, const double* den_fixed,
                             double* grad, int abs_hash)
{
    uint64_t n_mlp = mlp_param_count(c);
    const double* hash = params + n_mlp;
    int n_in = n_inputs(c);
    int H = c->hidden_layers, Wd = c->width;
    int L = c->hash_levels, F = c->feats_per_level;
    uint64_t Tab = 1ull << c->log2_table;
    int n_pos = n_pos_features(c);
    double loss = 0.0;
    double scale = 1.0 / (3.0 * (double)T);

    /* Per-sample backward in parallel; gradient accumulation in sample order. */
    double* de_all = (double*)calloc((size_t)T * n_pos, sizeof(double));
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    double* mlp_part = (double*)calloc((size_t)nthreads * n_mlp, sizeof(double));
    double* loss_part = (double*)calloc((size_t)T, sizeof(double));

#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double* g = mlp_part + (size_t)tid * n_mlp;
        double e[1024];
        double pre[MAX_LAYERS * MAX_WIDTH], act[MAX_LAYERS * MAX_WIDTH];
        double delta[MAX_WIDTH], delta_prev[MAX_WIDTH > 1024 ? MAX_WIDTH : 1024];
        double dabs[MAX_WIDTH], dabs_prev[MAX_WIDTH > 1024 ? MAX_WIDTH : 1024];
#pragma omp for schedule(static)
        for (int64_t t = 0; t < (int64_t)T; t++) {
            if (!gout && !(recs[t].flags & 1u)) continue;
            double z[3];
            encode(c, hash, &recs[t], dirs + 3 * t, e);
            mlp_forward(c, params, e, pre, act, z);
            double dz[3], dzabs[3];
            double lt = 0.0;
            for (int k = 0; k < 3; k++) {
                int vis = c->output == 1;
                int clamped = !vis && !(z[k] <= c->z_clamp);
                double nv = output_act(c, z[k]);
                double dn;
                if (gout) {
                    lt += gout[3 * t + k] * nv;
                    dn = gout[3 * t + k];
                } else if (vis) {
                    /* visibility: plain L2, (f - V)^2 */
                    double f = targets[3 * t + k];
                    lt += (f - nv) * (f - nv) * scale;
                    dn = -2.0 * (f - nv) * scale;
                } else {
                    double f = targets[3 * t + k];
                    double den = den_fixed ? den_fixed[3 * t + k] : nv * nv + c->loss_eps; /* sg(n)^2 + eps */
                    lt += (f - nv) * (f - nv) / den * scale;
                    dn = -2.0 * (f - nv) / den * scale;
                }
                /* dn/dz: exp' = n (0 above the clamp), sigmoid' = V (1 - V) */
                dz[k] = vis ? dn * nv * (1.0 - nv) : (clamped ? 0.0 : dn * nv);
                /* abs mode: the same with |f| + |n| in place of f - n (the scale of f - n's rounding) */
                if (abs_hash && !gout) {
                    double f = targets[3 * t + k];
                    double den = vis ? 1.0 : nv * nv + c->loss_eps;
                    double dna = 2.0 * (fabs(f) + fabs(nv)) / den * scale;
                    dzabs[k] = vis ? dna * nv * (1.0 - nv) : (clamped ? 0.0 : dna * nv);
                } else {
                    dzabs[k] = fabs(dz[k]);
                }
            }
            loss_part[t] = lt;
            /* Walk the layers backwards: delta = dL/d(pre-activation). */
            for (int k = 0; k < 3; k++) {
                delta[k] = dz[k];
                dabs[k] = dzabs[k];
            }
            int out = 3;
            uint64_t off = n_mlp;
            for (int l = H; l >= 0; l--) {
                int in = l == 0 ? n_in : Wd;
                off -= (uint64_t)out * in + out;
                const double* Wl = params + off;
                double* gW = g + off;
                double* gb = gW + (uint64_t)out * in;
                const double* x = l == 0 ? e : act + (l - 1) * MAX_WIDTH;
                for (int o = 0; o < out; o++) {
                    gb[o] += delta[o];
                    for (int i = 0; i < in; i++) gW[(uint64_t)o * in + i] += delta[o] * x[i];
                }
                for (int i = 0; i < in; i++) {
                    double s = 0.0, sa = 0.0;
                    for (int o = 0; o < out; o++) {
                        s += Wl[(uint64_t)o * in + i] * delta[o];
                        sa += fabs(Wl[(uint64_t)o * in + i]) * dabs[o];
                    }
                    delta_prev[i] = s;
                    dabs_prev[i] = sa;
                }
                if (l > 0) {
                    for (int i = 0; i < in; i++) {
                        const int on = pre[(l - 1) * MAX_WIDTH + i] > 0.0;
                        delta[i] = on ? delta_prev[i] : 0.0;
                        dabs[i] = on ? dabs_prev[i] : 0.0;
                    }
                } else {
                    for (int i = 0; i < n_pos; i++)
                        de_all[(size_t)t * n_pos + i] = abs_hash ? dabs_prev[i] : delta_prev[i];
                }
                out = in;
            }
        }
    }
    for (int th = 0; th < nthreads; th++)
        for (uint64_t i = 0; i < n_mlp; i++) grad[i] += mlp_part[(size_t)th * n_mlp + i];
    for (uint64_t t = 0; t < T; t++) loss += loss_part[t];

    /* Hash-grid features: dL/dtable[l][idx][f] += w_corner * dL/de[l*F + f]. */
    if (c->pos_encoding == 1) {
        double* gh = grad + n_mlp;
        for (uint64_t t = 0; t < T; t++) {
            if (!gout && !(recs[t].flags & 1u)) continue;
            for (int l = 0; l < L; l++) {
                uint32_t idx[8];
                double wts[8];
                orc_hash_level(c, l, recs[t].p, idx, wts);
                for (int corner = 0; corner < 8; corner++)
                    for (int f = 0; f < F; f++) {
                        double contrib = wts[corner] * de_all[(size_t)t * n_pos + l * F + f];
                        gh[((uint64_t)l * Tab + idx[corner]) * F + f] += abs_hash ? fabs(contrib) : contrib;
                    }
            }
        }
    }
    free(de_all);
    free(mlp_part);
    free(loss_part);
    return loss;
}

double orc_train_loss_grad(const o_cfg* c, const double* params, const o_record* recs, const float* dirs,
                           const double* targets, uint64_t T, const double* den_fixed, double* grad)
{
    return loss_grad_core(c, params, recs, dirs, targets, NULL, T, den_fixed, grad, 0);
}

/* orc_train_loss_grad with the hash-table part replaced by its running-error
 * scale: the same backward with every signed sum replaced by the sum of the
 * absolute values of its terms, i.e. |f| + |n| in place of f - n in dL/dn,
 * |W| in place of W through the layers (the ReLU masks kept), and
 * |w_corner| |dL/de| summed over records and corners.  An entry's rounding
 * error in any implementation of the backward is bounded by a small multiple
 * of this scale however much its terms cancel (test tolerances per entry).
 * When every weight and dL/dz is non-negative it equals the gradient.  The
 * MLP part is the ordinary gradient. */
double orc_train_loss_grad_abs(const o_cfg* c, const double* params, const o_record* recs, const float* dirs,
                               const double* targets, uint64_t T, double* grad)
{
    return loss_grad_core(c, params, recs, dirs, targets, NULL, T, NULL, grad, 1);
}

/* Gradient of sum_t sum_ch gout[t][ch] * n(record_t, dir_t) with respect to
 * every parameter (MLP and hash table), added into grad; returns the sum.
 * Every record counts (like orc_query, which ignores the valid flag). */
double orc_query_grad(const o_cfg* c, const double* params, const o_record* recs, const float* dirs,
                      const double* gout, uint64_t T, double* grad)
{
    return loss_grad_core(c, params, recs, dirs, NULL, gout, T, NULL, grad, 0);
}

/* ------------------------------------------------------------------------ */
/* Adam (Kingma & Ba 2015), bias-corrected, dense over all parameters       */
/* ------------------------------------------------------------------------ */

void orc_adam_step(uint64_t n, double* params, double* m, double* v, const double* g, uint32_t step, double lr,
                   double beta1, double beta2, double eps)
{
    double bc1 = 1.0 - pow(beta1, (double)step);
    double bc2 = 1.0 - pow(beta2, (double)step);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; i++) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
        double mhat = m[i] / bc1;
        double vhat = v[i] / bc2;
        params[i] -= lr * mhat / (sqrt(vhat) + eps);
    }
}

/* ------------------------------------------------------------------------ */
/* Frame metric: mean relative squared error over pixels and RGB            */
/* ------------------------------------------------------------------------ */

double orc_mrse(const double* img, const double* ref, uint64_t n_pixels, double eps)
{
    double s = 0.0;
    for (uint64_t i = 0; i < 3 * n_pixels; i++) {
        double d = img[i] - ref[i];
        s += d * d / (ref[i] * ref[i] + eps);
    }
    return n_pixels ? s / (3.0 * (double)n_pixels) : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Small entry points used by the pins                                      */
/* ------------------------------------------------------------------------ */

float orc_u01(uint32_t x)
{
    return u01(x);
}

int orc_trace(const uint8_t* blob, const float o[3], const float d[3], float* t)
{
    const o_header* hd = (const o_header*)blob;
    return trace_nearest(scene_prims(blob), hd->n_prims, o, d, t);
}

void orc_sample_bsdf(const o_record* rec, uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c3,
                     float wi[3], double w[3], int32_t* valid, uint32_t* rejected, uint32_t* lobe)
{
    o_sample s;
    sample_bsdf(rec, k0, k1, c0, c1, c3, &s);
    for (int k = 0; k < 3; k++) {
        wi[k] = s.wi[k];
        w[k] = s.w[k];
    }
    *valid = s.valid;
    *rejected = s.rejected;
    *lobe = s.lobe;
}

void orc_onb(const float n[3], float t[3], float b[3])
{
    onb(n, t, b);
}

void orc_trace_path(const uint8_t* blob, const float o[3], const float d[3], uint32_t k0, uint32_t k1, uint32_t c0,
                    uint32_t c1, uint32_t max_depth, double L[3])
{
    uint64_t sg = SIG_INIT;
    trace_path(blob, o, d, k0, k1, c0, c1, max_depth, L, &sg, NULL);
}

/* One NEE sample at a shading record (light mode 1 machinery, for the
 * pins): adds the weighted contribution into out, returns the decision
 * word. */
uint32_t orc_nee_sample(const uint8_t* blob, const o_record* rec, uint32_t n_b, uint32_t k0, uint32_t k1, uint32_t c0,
                        uint32_t c1, uint32_t c3, double out[3])
{
    o_lights lights;
    collect_lights(blob, &lights);
    return nee_sample(blob, &lights, rec, n_b, k0, k1, c0, c1, c3, out);
}

void orc_bsdf_eval(const o_record* rec, const float wi[3], double fcos[3], double* pdf)
{
    bsdf_eval(rec, wi, fcos, pdf);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
