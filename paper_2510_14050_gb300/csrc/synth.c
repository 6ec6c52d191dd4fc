/*
 * Seeded synthetic packet-window generator (host C, pthreads).
 *
 * This module produces the (src, dst) uint32 packet pairs that both the CPU
 * oracle and the CUDA library consume.  It contains none of the method's
 * arithmetic (no traffic matrix, no aggregation, no statistics): it only
 * draws addresses.  The workloads stand in for the Graph Challenge's
 * synthetic 2^30-packet data set (Sec. V "Dataset"), which is not available.
 *
 * Random numbers.  Every draw is a pure function of (seed, config, window,
 * purpose, sample, attempt): the SplitMix64 output function (Steele, Lea and
 * Flood, OOPSLA 2014) is evaluated at a counter, so results do not depend on
 * the thread count or on the order windows are produced in.
 *
 * Zipf(s) over {1..N}: rejection-inversion (Hormann and Derflinger, "Rejection-
 * inversion to generate variates from monotone discrete distributions", ACM
 * TOMACS 1996), exact for any N up to 2^32 and any s > 0.
 *
 * Rank -> address: addr(k) = (k - 1) * 0x9E3779B1 mod 2^32 (Knuth's odd
 * multiplicative constant, a bijection on 32-bit integers).
 *
 * Build with -ffp-contract=off so that x86-64 and aarch64 evaluate the same
 * floating-point expressions.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN64 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Output number i of the SplitMix64 sequence whose state starts at `key`. */
static inline uint64_t ctr_u64(uint64_t key, uint64_t i) {
    return mix64(key + (i + 1) * GOLDEN64);
}

/* A stream key for (seed, config, window, purpose). */
static uint64_t stream_key(uint64_t seed, int cfg, uint64_t window, uint32_t purpose) {
    uint64_t k = mix64(seed ^ 0x5DEECE66DULL);
    k = mix64(k ^ ((uint64_t)(uint32_t)cfg << 40) ^ ((uint64_t)purpose << 56));
    k = mix64(k + window * GOLDEN64);
    return k;
}

/* Uniform double in [0, 1) with 53 random bits. */
static inline double u01(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

static inline uint32_t rank_to_addr(uint64_t k) { return (uint32_t)((k - 1) * 0x9E3779B1ULL); }

/* ---------------------------------------------------------------- Zipf --- */

typedef struct {
    double s, one_minus_s;
    double n;              /* N as a double */
    double h_lo;           /* H(1.5) - h(1): lower end of the inversion interval */
    double h_hi;           /* H(N + 0.5): upper end */
} zipf_t;

/* expm1(t)/t and log1p(t)/t, continuous at t = 0. */
static double expm1_over(double t) { return fabs(t) > 1e-8 ? expm1(t) / t : 1.0 + 0.5 * t; }
static double log1p_over(double t) { return fabs(t) > 1e-8 ? log1p(t) / t : 1.0 - 0.5 * t; }

/* H(x) = integral_1^x t^-s dt ; h(x) = x^-s ; H^-1. */
static double zipf_H(const zipf_t* z, double x) {
    double lx = log(x);
    return expm1_over(z->one_minus_s * lx) * lx;
}
static double zipf_h(const zipf_t* z, double x) { return exp(-z->s * log(x)); }
static double zipf_Hinv(const zipf_t* z, double y) {
    double t = y * z->one_minus_s;
    if (t < -1.0) t = -1.0; /* guards rounding at the lower end */
    return exp(log1p_over(t) * y);
}

static void zipf_init(zipf_t* z, double s, uint64_t n) {
    z->s = s;
    z->one_minus_s = 1.0 - s;
    z->n = (double)n;
    z->h_lo = zipf_H(z, 1.5) - 1.0;
    z->h_hi = zipf_H(z, z->n + 0.5);
}

/* One Zipf rank in {1..N}; draws come from stream (key, sample). */
static uint64_t zipf_draw(const zipf_t* z, uint64_t key, uint64_t sample) {
    uint64_t skey = mix64(key + sample * 0xD1B54A32D192ED03ULL);
    for (uint64_t attempt = 0;; ++attempt) {
        double u = z->h_hi + u01(ctr_u64(skey, attempt)) * (z->h_lo - z->h_hi);
        double x = zipf_Hinv(z, u);
        double kf = floor(x + 0.5);
        if (kf < 1.0) kf = 1.0;
        if (kf > z->n) kf = z->n;
        if (u >= zipf_H(z, kf + 0.5) - zipf_h(z, kf)) return (uint64_t)kf;
    }
}

/* ------------------------------------------------------------- configs --- */

enum {
    P_SIZE = 1, P_SRC = 2, P_DST = 3, P_BURST_LEN = 4, P_BURST_POS = 5, P_BURST_PAIR = 6,
    P_HH_DST = 7, P_SCAN = 8, P_SHUFFLE = 9, P_ARRIVAL = 10
};

/* Window sizes.  cfg 3: floor(2^(10+10u)) clamped to [2^10, 2^20];
 * cfg 5: uniform integer in [2^12, 2^17]; others: 2^17. */
int synth_window_sizes(int cfg, uint64_t seed, uint64_t first_window, uint64_t nwin, uint64_t* sizes) {
    for (uint64_t i = 0; i < nwin; ++i) {
        uint64_t w = first_window + i;
        uint64_t key = stream_key(seed, cfg, w, P_SIZE);
        if (cfg == 3) {
            double u = u01(ctr_u64(key, 0));
            double p = floor(exp2(10.0 + 10.0 * u));
            if (p < 1024.0) p = 1024.0;
            if (p > 1048576.0) p = 1048576.0;
            sizes[i] = (uint64_t)p;
        } else if (cfg == 5) {
            uint64_t span = (1ULL << 17) - (1ULL << 12) + 1;
            sizes[i] = (1ULL << 12) + ctr_u64(key, 0) % span;
        } else if (cfg >= 1 && cfg <= 4) {
            sizes[i] = 1ULL << 17;
        } else {
            return -1;
        }
    }
    return 0;
}

/* Background pairs with independent Zipf ranks for src and dst. */
static void fill_iid(const zipf_t* zs, const zipf_t* zd, uint64_t key_s, uint64_t key_d,
                     uint64_t first_sample, uint64_t n, uint32_t* src, uint32_t* dst) {
    for (uint64_t i = 0; i < n; ++i) {
        src[i] = rank_to_addr(zipf_draw(zs, key_s, first_sample + i));
        dst[i] = rank_to_addr(zipf_draw(zd, key_d, first_sample + i));
    }
}

typedef struct { uint64_t pos, idx, len; uint32_t s, d; } burst_t;

static int burst_cmp(const void* a, const void* b) {
    const burst_t* x = (const burst_t*)a;
    const burst_t* y = (const burst_t*)b;
    if (x->pos != y->pos) return x->pos < y->pos ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx ? 1 : 0);
}

/* cfg 2 / cfg 5 traffic: floor(0.05 P) packets belong to bursts of length
 * U{2..100} (last one clipped; a leftover of 1 joins the previous burst); each
 * burst repeats one fresh pair and sits contiguously at a uniform insertion
 * point among the P - B background packets. */
static int fill_bursty(int cfg, uint64_t seed, uint64_t w, uint64_t p, uint32_t* src, uint32_t* dst) {
    zipf_t zs, zd;
    zipf_init(&zs, 1.1, 1ULL << 20);
    zipf_init(&zd, 1.3, 1ULL << 22);
    uint64_t ks = stream_key(seed, cfg, w, P_SRC), kd = stream_key(seed, cfg, w, P_DST);
    uint64_t b_total = (uint64_t)floor(0.05 * (double)p);
    uint64_t m = p - b_total;

    uint64_t kl = stream_key(seed, cfg, w, P_BURST_LEN);
    uint64_t nb = 0, cap = b_total / 2 + 2;
    burst_t* bursts = (burst_t*)malloc(sizeof(burst_t) * cap);
    if (!bursts) return -2;
    uint64_t left = b_total, draw = 0;
    while (left > 0) {
        uint64_t len = 2 + ctr_u64(kl, draw++) % 99;
        if (len > left) len = left;
        if (len == 1 && nb > 0) {
            bursts[nb - 1].len += 1;
        } else {
            bursts[nb].len = len;
            bursts[nb].idx = nb;
            ++nb;
        }
        left -= len;
    }
    uint64_t kp = stream_key(seed, cfg, w, P_BURST_POS);
    uint64_t kbs = stream_key(seed, cfg, w, P_BURST_PAIR);
    uint64_t kbd = stream_key(seed, cfg, w, P_BURST_PAIR + 100);
    for (uint64_t b = 0; b < nb; ++b) {
        bursts[b].pos = ctr_u64(kp, b) % (m + 1);
        bursts[b].s = rank_to_addr(zipf_draw(&zs, kbs, b));
        bursts[b].d = rank_to_addr(zipf_draw(&zd, kbd, b));
    }
    qsort(bursts, nb, sizeof(burst_t), burst_cmp);

    uint64_t out = 0, bi = 0;
    for (uint64_t i = 0; i <= m; ++i) {
        while (bi < nb && bursts[bi].pos == i) {
            for (uint64_t t = 0; t < bursts[bi].len; ++t) {
                src[out] = bursts[bi].s;
                dst[out] = bursts[bi].d;
                ++out;
            }
            ++bi;
        }
        if (i < m) {
            fill_iid(&zs, &zd, ks, kd, i, 1, src + out, dst + out);
            ++out;
        }
    }
    free(bursts);
    return out == p ? 0 : -3;
}

#define HEAVY_HITTER_SRC 0xC0A80001u
#define SCAN_POOL 16777u

/* cfg 3 traffic: a heavy hitter sends floor(0.10 P) packets to Zipf(1.1)/2^24
 * destinations; k = max(1, floor(P / 2^14)) scanners from a pool of 16,777
 * source ranks each hit f ~ loguniform[16, 2^16] consecutive destinations
 * (total capped at 10% of P); the rest is iid Zipf(1.1)/2^24; the window is
 * then shuffled (Fisher-Yates on the window's own stream). */
static int fill_mixed(uint64_t seed, uint64_t w, uint64_t p, uint32_t* src, uint32_t* dst) {
    const int cfg = 3;
    zipf_t z;
    zipf_init(&z, 1.1, 1ULL << 24);
    uint64_t out = 0;

    uint64_t nh = (uint64_t)floor(0.10 * (double)p);
    uint64_t khd = stream_key(seed, cfg, w, P_HH_DST);
    for (uint64_t i = 0; i < nh; ++i) {
        src[out] = HEAVY_HITTER_SRC;
        dst[out] = rank_to_addr(zipf_draw(&z, khd, i));
        ++out;
    }

    uint64_t kscan = stream_key(seed, cfg, w, P_SCAN);
    uint64_t nscan = p >> 14;
    if (nscan < 1) nscan = 1;
    uint64_t budget = (uint64_t)floor(0.10 * (double)p);
    for (uint64_t j = 0; j < nscan && budget > 0; ++j) {
        uint32_t s = rank_to_addr((1ULL << 24) + 1 + ctr_u64(kscan, 3 * j) % SCAN_POOL);
        uint64_t f = (uint64_t)floor(exp2(4.0 + 12.0 * u01(ctr_u64(kscan, 3 * j + 1))));
        if (f > budget) f = budget;
        uint32_t base = (uint32_t)ctr_u64(kscan, 3 * j + 2);
        for (uint64_t t = 0; t < f; ++t) {
            src[out] = s;
            dst[out] = base + (uint32_t)t;
            ++out;
        }
        budget -= f;
    }

    uint64_t ks = stream_key(seed, cfg, w, P_SRC), kd = stream_key(seed, cfg, w, P_DST);
    fill_iid(&z, &z, ks, kd, 0, p - out, src + out, dst + out);

    uint64_t ksh = stream_key(seed, cfg, w, P_SHUFFLE);
    for (uint64_t i = p; i > 1; --i) {
        uint64_t j = ctr_u64(ksh, i) % i;
        uint32_t a = src[i - 1]; src[i - 1] = src[j]; src[j] = a;
        uint32_t b = dst[i - 1]; dst[i - 1] = dst[j]; dst[j] = b;
    }
    return 0;
}

static int fill_window(int cfg, uint64_t seed, uint64_t w, uint64_t p, uint32_t* src, uint32_t* dst) {
    if (p == 0) return 0;
    if (cfg == 1 || cfg == 4) {
        zipf_t z;
        if (cfg == 1) zipf_init(&z, 1.2, 1ULL << 16);
        else zipf_init(&z, 1.05, 1ULL << 32);
        fill_iid(&z, &z, stream_key(seed, cfg, w, P_SRC), stream_key(seed, cfg, w, P_DST), 0, p, src, dst);
        return 0;
    }
    if (cfg == 2 || cfg == 5) return fill_bursty(cfg, seed, w, p, src, dst);
    if (cfg == 3) return fill_mixed(seed, w, p, src, dst);
    return -1;
}

typedef struct {
    int cfg;
    uint64_t seed, first_window, nwin;
    const uint64_t* offsets;
    uint32_t *src, *dst;
    uint64_t next;            /* shared work counter */
    pthread_mutex_t lock;
    int status;
} job_t;

static void* worker(void* arg) {
    job_t* j = (job_t*)arg;
    for (;;) {
        pthread_mutex_lock(&j->lock);
        uint64_t i = j->next++;
        pthread_mutex_unlock(&j->lock);
        if (i >= j->nwin) break;
        uint64_t a = j->offsets[i] - j->offsets[0], b = j->offsets[i + 1] - j->offsets[0];
        int rc = fill_window(j->cfg, j->seed, j->first_window + i, b - a, j->src + a, j->dst + a);
        if (rc != 0) {
            pthread_mutex_lock(&j->lock);
            j->status = rc;
            pthread_mutex_unlock(&j->lock);
        }
    }
    return NULL;
}

/* Fill windows [first_window, first_window + nwin) of a config.  offsets has
 * nwin + 1 entries (window i occupies [offsets[i], offsets[i+1]) relative to
 * offsets[0]); src and dst point at the slot of offsets[0]. */
int synth_fill(int cfg, uint64_t seed, uint64_t first_window, uint64_t nwin, const uint64_t* offsets,
               uint32_t* src, uint32_t* dst, int nthreads) {
    if (cfg < 1 || cfg > 5) return -1;
    job_t j;
    memset(&j, 0, sizeof(j));
    j.cfg = cfg; j.seed = seed; j.first_window = first_window; j.nwin = nwin;
    j.offsets = offsets; j.src = src; j.dst = dst;
    pthread_mutex_init(&j.lock, NULL);
    if (nthreads < 1) nthreads = 1;
    if ((uint64_t)nthreads > nwin) nthreads = nwin ? (int)nwin : 1;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nthreads);
    if (!th) return -2;
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, worker, &j);
    worker(&j);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&j.lock);
    return j.status;
}

/* Zipf ranks alone (for distribution tests of the sampler). */
int synth_zipf_ranks(double s, uint64_t n, uint64_t seed, uint64_t count, uint64_t* out) {
    if (!(s > 0.0) || n < 1) return -1;
    zipf_t z;
    zipf_init(&z, s, n);
    uint64_t key = stream_key(seed, 0, 0, 77);
    for (uint64_t i = 0; i < count; ++i) out[i] = zipf_draw(&z, key, i);
    return 0;
}

/* Poisson arrivals: t_i = t_{i-1} + Exp(rate), t_{-1} = 0 (seconds). */
int synth_arrivals(uint64_t seed, double rate, uint64_t n, double* t) {
    if (!(rate > 0.0)) return -1;
    uint64_t key = stream_key(seed, 5, 0, P_ARRIVAL);
    double acc = 0.0;
    for (uint64_t i = 0; i < n; ++i) {
        acc += -log1p(-u01(ctr_u64(key, i))) / rate;
        t[i] = acc;
    }
    return 0;
}
