/*
 * Seeded synthetic event-camera streams: the input fixtures shared by the
 * tests, the oracle and the benchmark.  This file holds none of the ESI
 * arithmetic (no integration, decay, clamp or mapping); it only models a
 * sensor that produces events.
 *
 * Sensor model (the ideal event camera of Sec. III-A, Eq. 1): each pixel keeps
 * a reference log intensity ref; it emits +1 whenever L(t) >= ref + C_p (then
 * ref += C_p) and -1 whenever L(t) <= ref - C_p (then ref -= C_p).  C_p is the
 * pixel's own threshold (mismatch around C_mean).  Crossing times are found on
 * monotone pieces of L (bisection, analytic inversion or linear interpolation
 * between samples) and rounded to integer microseconds.  Independent sensor
 * noise is a Poisson process per pixel with random polarity; hot pixels are
 * Poisson processes at 1-20 kHz.
 *
 * Scenes:
 *   0  sinusoid L = ln(mean + amp(y) sin(2 pi f (x - v t))) translating along x,
 *      amplitude growing linearly with the row y
 *   1  Gaussian blobs in log intensity, linear motion with toroidal wrap
 *   2  rotating checkerboard (edges as short ramps), bursts of global flicker,
 *      hot pixels
 *
 * Output order: non-decreasing t; ties broken by pixel index y*W + x, then by
 * emission order within the pixel.  Every random number comes from a
 * splitmix64 stream keyed by (seed, pixel) or (seed, object), so the output is
 * independent of the number of threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int64_t t;
    uint16_t x;
    uint16_t y;
    int8_t p;
    uint8_t pad[3];
} syn_event;

#define SYN_MAX_BURSTS 8

typedef struct {
    int32_t kind;
    int32_t W, H;
    int32_t n_blobs;
    double duration_s;
    int64_t t0_us;
    uint64_t seed;
    double C_mean, C_rel_sigma;
    double noise_hz;
    /* scene 0 */
    double sin_mean, sin_amp, sin_freq_cpx, sin_speed_pxs;
    /* scene 1 */
    double blob_sigma_min, blob_sigma_max, blob_speed_min, blob_speed_max;
    double blob_amp_min, blob_amp_max;
    /* scene 2 */
    double checker_px, rot_rad_s, checker_log_contrast, edge_px;
    double flicker_hz, flicker_log_depth, flicker_ramp_s;
    int32_t n_bursts, _pad0;
    double burst_start_s[SYN_MAX_BURSTS], burst_len_s[SYN_MAX_BURSTS];
    double hot_frac, hot_rate_min, hot_rate_max, hot_pos_prob;
    double sin_phase_px;
    /* thinning: keep each generated event with this probability (0 or >= 1:
       keep all), from a per-pixel generator of its own */
    double keep_prob;
} syn_scene;

/* ---------------------------------------------------------------- RNG */
static inline uint64_t sm64(uint64_t *s)
{
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static inline double u01(uint64_t *s) { return (double)(sm64(s) >> 11) * (1.0 / 9007199254740992.0); }
static inline double nrm(uint64_t *s)
{
    double a = u01(s), b = u01(s);
    if (a < 1e-300) a = 1e-300;
    return sqrt(-2.0 * log(a)) * cos(6.283185307179586 * b);
}
static uint64_t key_state(uint64_t seed, uint64_t a, uint64_t b)
{
    uint64_t s = seed ^ (a * 0xD1B54A32D192ED03ull) ^ (b * 0x8CB92BA72F3D8DD7ull);
    sm64(&s);
    sm64(&s);
    return s;
}

/* ------------------------------------------------ per-pixel event lists */
typedef struct {
    double t;   /* seconds from t0 */
    int8_t p;
    int32_t seq;
} pev;

typedef struct {
    pev *a;
    int64_t n, cap;
} pevbuf;

static void pb_push(pevbuf *b, double t, int p)
{
    if (b->n == b->cap) {
        b->cap = b->cap ? b->cap * 2 : 64;
        b->a = (pev *)realloc(b->a, (size_t)b->cap * sizeof(pev));
    }
    b->a[b->n].t = t;
    b->a[b->n].p = (int8_t)p;
    b->a[b->n].seq = (int32_t)b->n;
    b->n++;
}

static int pev_cmp(const void *x, const void *y)
{
    const pev *a = (const pev *)x, *b = (const pev *)y;
    if (a->t < b->t) return -1;
    if (a->t > b->t) return 1;
    return (a->seq > b->seq) - (a->seq < b->seq);
}

/* Poisson process of rate hz on [0, T); polarity +1 with probability pp. */
static void poisson(pevbuf *b, uint64_t *rs, double hz, double T, double pp)
{
    if (hz <= 0.0) return;
    double t = 0.0;
    for (;;) {
        double u = u01(rs);
        t += -log(1.0 - u) / hz;
        if (t >= T) break;
        pb_push(b, t, u01(rs) < pp ? 1 : -1);
    }
}

static double pixel_threshold(const syn_scene *sc, uint64_t *rs)
{
    double c = sc->C_mean * (1.0 + sc->C_rel_sigma * nrm(rs));
    if (c < 0.3 * sc->C_mean) c = 0.3 * sc->C_mean;
    return c;
}

/* ---------------------------------------------------------- scene 0 */
/* amplitude grows linearly down the rows: amp(y) = sin_amp (y + 0.5) / H */
static double s0_L(const syn_scene *sc, double amp, double x, double t)
{
    double th = 6.283185307179586 * sc->sin_freq_cpx * (x + sc->sin_phase_px - sc->sin_speed_pxs * t);
    return log(sc->sin_mean + amp * sin(th));
}

static void scene0_pixel(const syn_scene *sc, int x, int y, uint64_t *rs, pevbuf *b)
{
    double amp = sc->sin_amp * (y + 0.5) / sc->H;
    const double PI = 3.141592653589793;
    double T = sc->duration_s;
    double Cp = pixel_threshold(sc, rs);
    double f = sc->sin_freq_cpx, v = sc->sin_speed_pxs;
    double om = 2.0 * PI * f * v;     /* rad/s, theta decreases in time */
    double ref = s0_L(sc, amp, x, 0.0);
    double t = 0.0;
    while (t < T) {
        double th = 2.0 * PI * f * (x + sc->sin_phase_px - v * t);
        double n = floor((th - 0.5 * PI) / PI);
        double the = 0.5 * PI + n * PI;
        if (the >= th - 1e-12) the -= PI;
        double tb = t + (th - the) / om;
        if (tb > T) tb = T;
        double La = s0_L(sc, amp, x, t), Lb = s0_L(sc, amp, x, tb);
        int rising = Lb > La;
        for (;;) {
            double lvl = rising ? ref + Cp : ref - Cp;
            if (rising ? (lvl > Lb) : (lvl < Lb)) break;
            ref = lvl;
            double lo = t, hi = tb;
            for (int it = 0; it < 60; ++it) {
                double mid = 0.5 * (lo + hi);
                double Lm = s0_L(sc, amp, x, mid);
                if (rising ? (Lm < lvl) : (Lm > lvl)) lo = mid; else hi = mid;
            }
            pb_push(b, hi, rising ? 1 : -1);
        }
        t = tb;
    }
}

/* ---------------------------------------------------------- scene 1 */
typedef struct {
    double cx, cy, vx, vy, sigma, amp;
} blob;

typedef struct {
    double tc, st, a;   /* centre time, temporal sigma, amplitude */
} bump;

static int bump_cmp(const void *x, const void *y)
{
    const bump *a = (const bump *)x, *b = (const bump *)y;
    double sa = a->tc - 4.0 * a->st, sb = b->tc - 4.0 * b->st;
    return (sa > sb) - (sa < sb);
}

static void make_blobs(const syn_scene *sc, blob *bl)
{
    for (int i = 0; i < sc->n_blobs; ++i) {
        uint64_t s = key_state(sc->seed, 0xB10Bull, (uint64_t)i);
        bl[i].cx = u01(&s) * sc->W;
        bl[i].cy = u01(&s) * sc->H;
        bl[i].sigma = sc->blob_sigma_min + u01(&s) * (sc->blob_sigma_max - sc->blob_sigma_min);
        double sp = sc->blob_speed_min + u01(&s) * (sc->blob_speed_max - sc->blob_speed_min);
        double dir = 6.283185307179586 * u01(&s);
        bl[i].vx = sp * cos(dir);
        bl[i].vy = sp * sin(dir);
        double a = sc->blob_amp_min + u01(&s) * (sc->blob_amp_max - sc->blob_amp_min);
        bl[i].amp = (u01(&s) < 0.5) ? a : -a;
    }
}

static double bumps_L(const bump *bs, int nb, double t)
{
    double L = 0.0;
    for (int j = 0; j < nb; ++j) {
        double z = (t - bs[j].tc) / bs[j].st;
        if (z > -6.0 && z < 6.0) L += bs[j].a * exp(-0.5 * z * z);
    }
    return L;
}

static void scene1_pixel(const syn_scene *sc, const blob *bl, int x, int y,
                         uint64_t *rs, pevbuf *b, bump **scratch, int *scap)
{
    double T = sc->duration_s;
    double Cp = pixel_threshold(sc, rs);
    double px = x + 0.5, py = y + 0.5;
    int nb = 0;
    for (int i = 0; i < sc->n_blobs; ++i) {
        const blob *o = &bl[i];
        double v2 = o->vx * o->vx + o->vy * o->vy;
        double spd = sqrt(v2);
        double r4 = 4.0 * o->sigma;
        double xa = o->cx, xb = o->cx + o->vx * T, ya = o->cy, yb = o->cy + o->vy * T;
        double xmin = fmin(xa, xb), xmax = fmax(xa, xb), ymin = fmin(ya, yb), ymax = fmax(ya, yb);
        int k0 = (int)ceil((-r4 - xmax) / sc->W), k1 = (int)floor((sc->W + r4 - xmin) / sc->W);
        int l0 = (int)ceil((-r4 - ymax) / sc->H), l1 = (int)floor((sc->H + r4 - ymin) / sc->H);
        for (int k = k0; k <= k1; ++k)
            for (int l = l0; l <= l1; ++l) {
                double qx = px - (o->cx + k * sc->W), qy = py - (o->cy + l * sc->H);
                double qv = qx * o->vx + qy * o->vy;
                double tc = qv / v2;
                double d2 = qx * qx + qy * qy - qv * qv / v2;
                double st = o->sigma / spd;
                if (tc + 4.0 * st < 0.0 || tc - 4.0 * st > T) continue;
                double a = o->amp * exp(-0.5 * d2 / (o->sigma * o->sigma));
                if (fabs(a) < 0.02) continue;
                if (nb == *scap) {
                    *scap = *scap ? *scap * 2 : 16;
                    *scratch = (bump *)realloc(*scratch, (size_t)*scap * sizeof(bump));
                }
                (*scratch)[nb].tc = tc;
                (*scratch)[nb].st = st;
                (*scratch)[nb].a = a;
                nb++;
            }
    }
    if (nb == 0) return;
    bump *bs = *scratch;
    qsort(bs, nb, sizeof(bump), bump_cmp);
    double ref = bumps_L(bs, nb, 0.0);
    /* walk merged support intervals; inside, sample and interpolate */
    int i = 0;
    while (i < nb) {
        double s0 = bs[i].tc - 4.0 * bs[i].st, e0 = bs[i].tc + 4.0 * bs[i].st;
        double stmin = bs[i].st;
        int j = i + 1;
        while (j < nb && bs[j].tc - 4.0 * bs[j].st <= e0) {
            double e = bs[j].tc + 4.0 * bs[j].st;
            if (e > e0) e0 = e;
            if (bs[j].st < stmin) stmin = bs[j].st;
            ++j;
        }
        if (s0 < 0.0) s0 = 0.0;
        if (e0 > T) e0 = T;
        double h = stmin / 8.0;
        if (h < 1e-6) h = 1e-6;
        double ta = s0, La = bumps_L(bs, nb, ta);
        while (ta < e0) {
            double tb = ta + h;
            if (tb > e0) tb = e0;
            double Lb = bumps_L(bs, nb, tb);
            while (Lb >= ref + Cp) {
                ref += Cp;
                double f = (Lb != La) ? (ref - La) / (Lb - La) : 1.0;
                if (f < 0.0) f = 0.0;
                pb_push(b, ta + f * (tb - ta), 1);
            }
            while (Lb <= ref - Cp) {
                ref -= Cp;
                double f = (Lb != La) ? (ref - La) / (Lb - La) : 1.0;
                if (f < 0.0) f = 0.0;
                pb_push(b, ta + f * (tb - ta), -1);
            }
            ta = tb;
            La = Lb;
        }
        i = j;
    }
}

/* ---------------------------------------------------------- scene 2 */
typedef struct {
    double ts, tau, delta;
} ramp;

static int ramp_cmp(const void *x, const void *y)
{
    const ramp *a = (const ramp *)x, *b = (const ramp *)y;
    return (a->ts > b->ts) - (a->ts < b->ts);
}

static void add_ramp(ramp **rp, int *n, int *cap, double ts, double tau, double delta)
{
    if (*n == *cap) {
        *cap = *cap ? *cap * 2 : 64;
        *rp = (ramp *)realloc(*rp, (size_t)*cap * sizeof(ramp));
    }
    (*rp)[*n].ts = ts;
    (*rp)[*n].tau = tau;
    (*rp)[*n].delta = delta;
    (*n)++;
}

/* all alpha = base + 2 pi j inside (alo, ahi] */
static void angles_in(double base, double alo, double ahi, double *out, int *n, int max)
{
    const double TWO_PI = 6.283185307179586;
    double j0 = ceil((alo - base) / TWO_PI - 1e-12);
    for (double j = j0;; j += 1.0) {
        double a = base + j * TWO_PI;
        if (a <= alo) continue;
        if (a > ahi || *n >= max) break;
        out[(*n)++] = a;
    }
}

static void scene2_pixel(const syn_scene *sc, int x, int y, uint64_t *rs, pevbuf *b,
                         ramp **rp, int *rcap)
{
    double T = sc->duration_s;
    double Cp = pixel_threshold(sc, rs);
    double cx = 0.5 * sc->W, cy = 0.5 * sc->H;
    double dx = x + 0.5 - cx, dy = y + 0.5 - cy;
    double r = sqrt(dx * dx + dy * dy);
    double phi = atan2(dy, dx);
    double om = sc->rot_rad_s, s = sc->checker_px, cl = sc->checker_log_contrast;
    int nr = 0;
    /* initial parity */
    double u0 = r * cos(phi), v0 = r * sin(phi);
    long par = ((long)floor(u0 / s) + (long)floor(v0 / s)) & 1L;
    double level = par ? 0.5 * cl : -0.5 * cl;
    if (r > 0.5 && om > 0.0) {
        double alo = phi - om * T, ahi = phi;
        int mmax = (int)floor(r / s);
        double angs[64];
        for (int m = -mmax; m <= mmax; ++m) {
            double c = m * s / r;
            if (c <= -1.0 || c >= 1.0) continue;
            /* u = r cos(alpha) = m s at alpha = +-acos(c);
               v = r sin(alpha) = m s at alpha = asin(c), pi - asin(c) */
            double base[4] = {acos(c), -acos(c), asin(c), 3.141592653589793 - asin(c)};
            for (int q = 0; q < 4; ++q) {
                int vline = q >= 2;
                int na = 0;
                angles_in(base[q], alo, ahi, angs, &na, 64);
                for (int k = 0; k < na; ++k) {
                    double a = angs[k];
                    double speed = r * om * (vline ? fabs(cos(a)) : fabs(sin(a)));
                    double tau = speed > 0.0 ? sc->edge_px / speed : 0.02;
                    if (tau < 2e-6) tau = 2e-6;
                    if (tau > 0.02) tau = 0.02;
                    double tc = (phi - a) / om;
                    add_ramp(rp, &nr, rcap, tc - 0.5 * tau, tau, 0.0); /* delta set below */
                }
            }
        }
        qsort(*rp, nr, sizeof(ramp), ramp_cmp);
        /* every grid-line crossing flips the cell parity */
        double lv = level;
        for (int k = 0; k < nr; ++k) {
            double to = (lv > 0.0) ? -0.5 * cl : 0.5 * cl;
            (*rp)[k].delta = to - lv;
            lv = to;
        }
    }
    /* flicker bursts: global square modulation with ramps */
    for (int bi = 0; bi < sc->n_bursts && bi < SYN_MAX_BURSTS; ++bi) {
        double hp = 0.5 / sc->flicker_hz, d = sc->flicker_log_depth;
        double t = sc->burst_start_s[bi], te = t + sc->burst_len_s[bi];
        double cur = 0.0;
        int sgn = 1;
        while (t < te) {
            double to = 0.5 * d * sgn;
            add_ramp(rp, &nr, rcap, t, sc->flicker_ramp_s, to - cur);
            cur = to;
            sgn = -sgn;
            t += hp;
        }
        add_ramp(rp, &nr, rcap, te, sc->flicker_ramp_s, -cur);
    }
    if (nr > 0) qsort(*rp, nr, sizeof(ramp), ramp_cmp);
    double L = level, ref = level, tprev_end = -1.0;
    for (int k = 0; k < nr; ++k) {
        ramp *q = &(*rp)[k];
        double ts = q->ts > tprev_end ? q->ts : tprev_end;
        double de = q->delta;
        if (de == 0.0) continue;
        double Le = L + de, em1 = expm1(de);
        for (;;) {
            double lvl = de > 0.0 ? ref + Cp : ref - Cp;
            if (de > 0.0 ? lvl > Le : lvl < Le) break;
            ref = lvl;
            double f = expm1(lvl - L) / em1;
            double te = ts + f * q->tau;
            if (te >= 0.0 && te < T) pb_push(b, te, de > 0.0 ? 1 : -1);
        }
        L = Le;
        tprev_end = ts + q->tau;
    }
    /* hot pixel */
    if (sc->hot_frac > 0.0 && u01(rs) < sc->hot_frac) {
        double lr = log(sc->hot_rate_min) + u01(rs) * (log(sc->hot_rate_max) - log(sc->hot_rate_min));
        poisson(b, rs, exp(lr), T, sc->hot_pos_prob);
    }
}

/* ------------------------------------------------------------ driver */
typedef struct {
    int64_t t;       /* microseconds from t0 */
    uint32_t pix;
    int8_t p;
} rowev;

typedef struct {
    rowev *a;
    int64_t n, cap;
} rowbuf;

syn_event *syn_generate(const syn_scene *sc, int64_t *n_out, int nthreads)
{
    int W = sc->W, H = sc->H;
    double T = sc->duration_s;
    int64_t Tus = (int64_t)llround(T * 1e6);
    rowbuf *rows = (rowbuf *)calloc((size_t)H, sizeof(rowbuf));
    blob *bl = NULL;
    if (sc->kind == 1) {
        bl = (blob *)calloc((size_t)(sc->n_blobs > 0 ? sc->n_blobs : 1), sizeof(blob));
        make_blobs(sc, bl);
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        pevbuf pb = {0};
        bump *bscr = NULL;
        int bcap = 0;
        ramp *rscr = NULL;
        int rcap = 0;
#pragma omp for schedule(dynamic, 1)
        for (int y = 0; y < H; ++y) {
            rowbuf *rb = &rows[y];
            for (int x = 0; x < W; ++x) {
                uint32_t pix = (uint32_t)y * (uint32_t)W + (uint32_t)x;
                uint64_t rs = key_state(sc->seed, 0x9191ull, pix);
                pb.n = 0;
                if (sc->kind == 0)
                    scene0_pixel(sc, x, y, &rs, &pb);
                else if (sc->kind == 1)
                    scene1_pixel(sc, bl, x, y, &rs, &pb, &bscr, &bcap);
                else
                    scene2_pixel(sc, x, y, &rs, &pb, &rscr, &rcap);
                poisson(&pb, &rs, sc->noise_hz, T, 0.5);
                if (pb.n > 1) qsort(pb.a, (size_t)pb.n, sizeof(pev), pev_cmp);
                const int thin = sc->keep_prob > 0.0 && sc->keep_prob < 1.0;
                uint64_t ks = key_state(sc->seed, 0x5151ull, pix);
                int64_t last = 0;
                for (int64_t i = 0; i < pb.n; ++i) {
                    if (thin && u01(&ks) >= sc->keep_prob) continue;
                    int64_t tu = (int64_t)llround(pb.a[i].t * 1e6);
                    if (tu < last) tu = last;
                    if (tu < 0 || tu > Tus) continue;
                    last = tu;
                    if (rb->n == rb->cap) {
                        rb->cap = rb->cap ? rb->cap * 2 : 256;
                        rb->a = (rowev *)realloc(rb->a, (size_t)rb->cap * sizeof(rowev));
                    }
                    rb->a[rb->n].t = tu;
                    rb->a[rb->n].pix = pix;
                    rb->a[rb->n].p = pb.a[i].p;
                    rb->n++;
                }
            }
        }
        free(pb.a);
        free(bscr);
        free(rscr);
    }
    /* stable counting sort by t; rows in order keep ties ordered by pixel */
    int64_t n = 0;
    for (int y = 0; y < H; ++y) n += rows[y].n;
    int64_t *cnt = (int64_t *)calloc((size_t)Tus + 2, sizeof(int64_t));
    for (int y = 0; y < H; ++y)
        for (int64_t i = 0; i < rows[y].n; ++i) cnt[rows[y].a[i].t + 1]++;
    for (int64_t i = 1; i <= Tus + 1; ++i) cnt[i] += cnt[i - 1];
    syn_event *out = (syn_event *)malloc((size_t)(n > 0 ? n : 1) * sizeof(syn_event));
    for (int y = 0; y < H; ++y) {
        for (int64_t i = 0; i < rows[y].n; ++i) {
            rowev *e = &rows[y].a[i];
            syn_event *o = &out[cnt[e->t]++];
            o->t = sc->t0_us + e->t;
            o->x = (uint16_t)(e->pix % (uint32_t)W);
            o->y = (uint16_t)(e->pix / (uint32_t)W);
            o->p = e->p;
            o->pad[0] = o->pad[1] = o->pad[2] = 0;
        }
        free(rows[y].a);
    }
    free(cnt);
    free(rows);
    free(bl);
    *n_out = n;
    return out;
}

void syn_free(void *p) { free(p); }

void syn_copy(const syn_event *src, int64_t n, void *dst)
{
    memcpy(dst, src, (size_t)n * sizeof(syn_event));
}
