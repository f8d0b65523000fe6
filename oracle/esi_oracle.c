/*
 * FP64 reference implementation ("oracle") of Event-based Single Integration.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load this file's library.  The CUDA
 * product path shares no code, header, table or constant with it.
 *
 * What it computes, in the paper's order and notation:
 *   - Alg. 2 (Sec. III-C): for every event e_i = (x_i, y_i, p_i, t_i), in the
 *     order it was pushed:  S += p_i C;  dt = t_i - T;  S *= d(dt);  T = t_i;
 *     S = min(max(S, S_min), S_max)   (the clamp of Eq. 13, applied per event
 *     as Alg. 2 places it inside the loop).
 *   - Eq. 4 (Sec. III-B): d(t) = max{(1 - k t)^b, 0}.  Read as
 *     max(1 - k t, 0)^b, so that d = 0 once k t >= 1 and d(0) = 1 (the
 *     printed form is undefined or amplifying for 1 - k t < 0 with
 *     non-integer or even b).
 *   - Eq. 14 (Sec. III-C): B = 255 (S - S_min) / (S_max - S_min), rounded
 *     half to even and saturated to [0, 255] (the paper does not say how it
 *     rounds).  With render_decay = 1 the value mapped is the decay view
 *     S * d(t_frame - T), which is not written back; with render_decay = 0 it
 *     is S as stored, as Alg. 2 renders it.
 *
 * Three methods share the event loop (argument `method`):
 *   0  Alg. 2 as above (the default).
 *   1  Alg. 1 (Sec. III-B): the same loop without the clamp of Eq. 13.  With
 *      k = 0 it is the plain integration of Eq. 2.
 *   2  Eq. 3 (Sec. III-B) with the exponential decay d(t) = exp(-k t):
 *      L(t) = C sum_{t_i <= t} p_i exp(-k (t - t_i)), no clamp.  Since
 *      exp(-k a) exp(-k b) = exp(-k (a + b)), the sum regroups exactly (up to
 *      rounding) into a per-pixel recurrence on (S, T) = (L(T), the last
 *      event time):  S <- S exp(-k (t_i - T)) + p_i C;  T <- t_i.  The event's
 *      own term enters undecayed, unlike Alg. 1 and 2.  b is not used.
 * For every method the render maps with Eq. 14 and saturates to [0, 255];
 * the decay view uses the method's own d.
 *
 * Diagnostics (Sec. III-B, Fig. 4): the noise-accumulation map ln(1 + |S|)
 * and per-pixel event counts.  Continuous-time output: S right after every
 * event.
 *
 * Other readings: polarity p > 0 counts +1, anything else -1 (Sec. III-A gives
 * p in {+1, -1}); events with x >= W or y >= H are dropped and counted, never
 * applied; time is int64 microseconds and k is given per second, so the
 * product k t uses k * 1e-6 per microsecond.  Events at one pixel must arrive
 * in non-decreasing time (the caller checks this).
 *
 * Precision: every state value and every intermediate is IEEE double.  Build
 * with -ffp-contract=off so that no multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>

/* Event record as laid out in memory: 16 bytes. */
typedef struct {
    int64_t t;   /* microseconds */
    uint16_t x;
    uint16_t y;
    int8_t p;    /* polarity */
    uint8_t pad[3];
} oracle_event;

/* Eq. 4 with the reading max(1 - k dt, 0)^b; dt in microseconds, k in 1/s. */
double oracle_decay(int64_t dt_us, double k_per_s, double b)
{
    double u = 1.0 - (k_per_s * 1e-6) * (double)dt_us;
    if (u > 0.0)
        return pow(u, b);
    return 0.0;
}

/* The decay of Eq. 3 read with d(t) = exp(-k t); dt in microseconds, k in 1/s. */
double oracle_decay_exp(int64_t dt_us, double k_per_s)
{
    return exp(-(k_per_s * 1e-6) * (double)dt_us);
}

/* The decay function of a method (Eq. 4 for Alg. 1 and 2, exp for Eq. 3). */
static double method_decay(int method, int64_t dt, double k_per_s, double b)
{
    if (method == 2)
        return oracle_decay_exp(dt, k_per_s);
    return oracle_decay(dt, k_per_s, b);
}

/* One pass of the event loop for one accepted event at pixel index pix. */
static void oracle_step(double *S, int64_t *T, int64_t pix, int8_t p, int64_t t,
                        double C, double k_per_s, double b, double s_min,
                        double s_max, int method)
{
    double pol = (p > 0) ? 1.0 : -1.0;
    double s = S[pix];
    if (method == 2) {
        /* Eq. 3 regrouped: L(t_i) = L(T) exp(-k (t_i - T)) + p_i C */
        s = s * oracle_decay_exp(t - T[pix], k_per_s);
        s = s + pol * C;
        T[pix] = t;
        S[pix] = s;
        return;
    }
    s = s + pol * C;                              /* S <- S + p C          */
    int64_t dt = t - T[pix];                      /* dt <- t - T           */
    s = s * oracle_decay(dt, k_per_s, b);         /* S <- S max{(1-k dt)^b,0} */
    T[pix] = t;                                   /* T <- t                */
    if (method == 0) {                            /* S <- min(max(S,Smin),Smax) */
        if (s < s_min) s = s_min;
        if (s > s_max) s = s_max;
    }
    S[pix] = s;
}

/*
 * Initialise the accumulation matrix S to 0 and the last-decay-time matrix T
 * to t_origin (Alg. 2 initialises both to zero; t_origin = 0 is the paper's
 * choice).
 */
void oracle_init(double *S, int64_t *T, int64_t P, int64_t t_origin)
{
    for (int64_t i = 0; i < P; ++i) {
        S[i] = 0.0;
        T[i] = t_origin;
    }
}

/*
 * The event loop (Alg. 2, Alg. 1 or Eq. 3 by `method`) over n events in push
 * order.  S and T (row-major, pixel
 * y*W + x) are updated in place.  Returns the number of events applied;
 * *dropped is increased by the number of out-of-range events.
 */
int64_t oracle_integrate(const oracle_event *ev, int64_t n, int W, int H,
                         double C, double k_per_s, double b, double s_min,
                         double s_max, int method, double *S, int64_t *T,
                         int64_t *dropped)
{
    int64_t applied = 0;
    for (int64_t i = 0; i < n; ++i) {
        const oracle_event *e = &ev[i];
        if ((int)e->x >= W || (int)e->y >= H) {
            *dropped += 1;
            continue;
        }
        int64_t pix = (int64_t)e->y * W + e->x;
        oracle_step(S, T, pix, e->p, e->t, C, k_per_s, b, s_min, s_max,
                    method);
        applied += 1;
    }
    return applied;
}

/* Eq. 14 for every pixel; render_decay selects the decay view (see header). */
void oracle_render(const double *S, const int64_t *T, int64_t P, double k_per_s,
                   double b, double s_min, double s_max, int render_decay,
                   int method, int64_t t_frame, uint8_t *B)
{
    for (int64_t i = 0; i < P; ++i) {
        double v = S[i];
        if (render_decay)
            v = v * method_decay(method, t_frame - T[i], k_per_s, b);
        double q = 255.0 * (v - s_min) / (s_max - s_min);
        double r = rint(q);
        if (r < 0.0) r = 0.0;
        if (r > 255.0) r = 255.0;
        B[i] = (uint8_t)r;
    }
}

/*
 * A sequence of M frames at non-decreasing times t_frames[w]: before frame w,
 * every not yet applied event with t <= t_frames[w] is applied in push order
 * (a frame at t shows the events with t_n <= t, the condition stated under
 * Eq. 5); then frame w is rendered into B + w * W * H.  Events after the last
 * frame time stay unapplied.  Returns the number of events consumed (applied
 * or dropped).
 */
int64_t oracle_replay(const oracle_event *ev, int64_t n, int W, int H,
                      double C, double k_per_s, double b, double s_min,
                      double s_max, int render_decay, int method,
                      const int64_t *t_frames, int64_t M, double *S, int64_t *T,
                      uint8_t *B, int64_t *dropped)
{
    int64_t P = (int64_t)W * H;
    int64_t i = 0;
    for (int64_t w = 0; w < M; ++w) {
        int64_t j = i;
        while (j < n && ev[j].t <= t_frames[w])
            ++j;
        oracle_integrate(ev + i, j - i, W, H, C, k_per_s, b, s_min, s_max,
                         method, S, T, dropped);
        i = j;
        oracle_render(S, T, P, k_per_s, b, s_min, s_max, render_decay, method,
                      t_frames[w], B + w * P);
    }
    return i;
}

/*
 * The noise-accumulation map of Fig. 4 (Sec. III-B): for every pixel the
 * absolute value of S, plus one, through the natural logarithm:
 * N = ln(1 + |S|).  Sec. III-B draws it for the plain integration of Eq. 2
 * over 2 s; any state may be passed.
 */
void oracle_noise_map(const double *S, int64_t P, double *N)
{
    for (int64_t i = 0; i < P; ++i)
        N[i] = log(1.0 + fabs(S[i]));
}

/*
 * Per-pixel event counts (the event-trigger rate of Sec. III-B times the
 * window): counts[y * W + x] = number of the n events at (x, y); events with
 * x >= W or y >= H are not counted.  counts is overwritten.
 */
void oracle_count_events(const oracle_event *ev, int64_t n, int W, int H,
                         uint32_t *counts)
{
    for (int64_t i = 0; i < (int64_t)W * H; ++i)
        counts[i] = 0;
    for (int64_t i = 0; i < n; ++i) {
        if ((int)ev[i].x >= W || (int)ev[i].y >= H)
            continue;
        counts[(int64_t)ev[i].y * W + ev[i].x] += 1;
    }
}

/*
 * Per-event states (continuous-time output): the event loop of `method` over
 * n events in push order, as oracle_integrate, writing out[i] = S of event
 * i's pixel right after event i is applied; NaN for an event outside the
 * sensor (never applied).  S and T are updated in place.
 */
void oracle_event_states(const oracle_event *ev, int64_t n, int W, int H,
                         double C, double k_per_s, double b, double s_min,
                         double s_max, int method, double *S, int64_t *T,
                         double *out)
{
    for (int64_t i = 0; i < n; ++i) {
        const oracle_event *e = &ev[i];
        if ((int)e->x >= W || (int)e->y >= H) {
            out[i] = NAN;
            continue;
        }
        int64_t pix = (int64_t)e->y * W + e->x;
        oracle_step(S, T, pix, e->p, e->t, C, k_per_s, b, s_min, s_max, method);
        out[i] = S[pix];
    }
}
