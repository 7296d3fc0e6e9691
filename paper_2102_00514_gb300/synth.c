/*
 * Seeded synthetic workload generator: coordinated-turn truth trajectories and
 * bearings-only measurements from two sensors (the simulated experiment of
 * Sec. 5; model of Eq. 4).
 *
 * This file produces INPUTS only. It is shared, as data, by the CUDA path and
 * by the CPU oracle, and holds none of the smoother's arithmetic (no
 * linearisation, no filtering, no smoothing). Its coordinated-turn propagation
 * is its own copy, used only to simulate the truth.
 *
 * Random numbers are counter based: every draw is a pure function of
 * (seed, trajectory, step, stream), hashed with SplitMix64 (Steele, Lea and
 * Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), so any
 * length or batch is reproducible and can be generated in any order. Normal
 * draws use the Box-Muller transform.
 *
 * Layouts: states are stored state-major, x[k*5 + i]; measurements y[k*2 + j].
 * Slot k = offsets[b] of trajectory b is its initial state x_0 (no
 * measurement; y there is set to 0).
 */
#include <math.h>
#include <stdint.h>

#define SYN_PI 3.14159265358979323846

/* stream ids of the counter-based generator */
enum {
    S_X0 = 0,        /* 0..4: initial truth state */
    S_Q = 8,         /* 8..12: process noise */
    S_R = 16,        /* 16..17: measurement noise */
    S_OMEGA0 = 24,   /* uniform truth turn rate */
    S_SENSOR = 25,   /* 25..28: sensor jitter */
    S_LENGTH = 32    /* trajectory length */
};

static uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

static uint64_t counter_hash(uint64_t seed, uint64_t traj, uint64_t step, uint64_t stream)
{
    uint64_t h = splitmix64(seed);
    h = splitmix64(h ^ traj);
    h = splitmix64(h ^ step);
    return splitmix64(h ^ stream);
}

/* uniform in the open interval (0, 1), 53 random bits, from sub-stream `sub` */
static double uniform_sub(uint64_t seed, uint64_t traj, uint64_t step, uint64_t sub)
{
    uint64_t h = counter_hash(seed, traj, step, sub);
    return ((double)(h >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

/* Every stream id s owns the two sub-streams 2s and 2s+1, so distinct stream
 * ids never share a draw. */
static double uniform01(uint64_t seed, uint64_t traj, uint64_t step, uint64_t stream)
{
    return uniform_sub(seed, traj, step, 2 * stream);
}

/* standard normal by Box-Muller from the two sub-streams of `stream` */
static double normal01(uint64_t seed, uint64_t traj, uint64_t step, uint64_t stream)
{
    double u1 = uniform_sub(seed, traj, step, 2 * stream);
    double u2 = uniform_sub(seed, traj, step, 2 * stream + 1);
    return sqrt(-2.0 * log(u1)) * cos(2.0 * SYN_PI * u2);
}

/* Coordinated-turn transition for the truth simulation. */
static void ct_propagate(const double x[5], double dt, double out[5])
{
    double w = x[4];
    double a = w * dt;
    double s = sin(a), cs = cos(a);
    double s_over_w, omc_over_w;
    if (fabs(a) < 1e-4) {
        double a2 = a * a;
        s_over_w = dt * (1.0 - a2 / 6.0 + a2 * a2 / 120.0);
        omc_over_w = dt * a * (0.5 - a2 / 24.0 + a2 * a2 / 720.0);
    } else {
        s_over_w = s / w;
        omc_over_w = (1.0 - cs) / w;
    }
    out[0] = x[0] + s_over_w * x[2] - omc_over_w * x[3];
    out[1] = x[1] + omc_over_w * x[2] + s_over_w * x[3];
    out[2] = cs * x[2] - s * x[3];
    out[3] = s * x[2] + cs * x[3];
    out[4] = w;
}

/*
 * Trajectory lengths T_b uniform on the integers [lo, hi].
 */
void synth_lengths(uint64_t seed, int64_t B, int64_t lo, int64_t hi, int64_t* T_out)
{
    for (int64_t b = 0; b < B; ++b) {
        double u = uniform01(seed, (uint64_t)b, 0, S_LENGTH);
        int64_t t = lo + (int64_t)floor(u * (double)(hi - lo + 1));
        if (t > hi) t = hi;
        T_out[b] = t;
    }
}

/*
 * Sensor positions per trajectory: base (s1x, s1y, s2x, s2y) plus, when
 * jitter > 0, an independent U(-jitter, jitter) offset on each coordinate.
 */
void synth_sensors(uint64_t seed, int64_t B, const double base[4], double jitter, double* sensors_out)
{
    for (int64_t b = 0; b < B; ++b)
        for (int i = 0; i < 4; ++i) {
            double off = 0.0;
            if (jitter > 0.0)
                off = jitter * (2.0 * uniform01(seed, (uint64_t)b, 0, S_SENSOR + i) - 1.0);
            sensors_out[b * 4 + i] = base[i] + off;
        }
}

/*
 * Truth and measurements.
 *   offsets[B+1]: state offsets (trajectory b owns states offsets[b]..offsets[b+1]-1)
 *   x0_mean[5], x0_std[5]: truth x_0 ~ N(x0_mean, diag(x0_std^2)), per trajectory
 *   omega0_halfwidth > 0: the truth turn rate of x_0 is instead U(-hw, hw)
 *   q_form 0: Q = diag(0, 0, q_c dt, q_c dt, q_w dt)
 *   q_form 1: continuous white acceleration, q_c [[dt^3/3, dt^2/2], [dt^2/2, dt]]
 *             per axis on (position, velocity), and q_w dt on the turn rate
 *   sensors[B or 1][4], sensors_per_traj selects which
 *   x_out[N][5], y_out[N][2]
 */
void synth_ct_bearings(uint64_t seed, int64_t B, const int64_t* offsets,
                       double dt, double q_c, double q_w, int q_form, double r_std,
                       const double x0_mean[5], const double x0_std[5], double omega0_halfwidth,
                       const double* sensors, int sensors_per_traj,
                       double* x_out, double* y_out)
{
    /* Cholesky factor of the per-axis (position, velocity) block of Q. */
    double l11 = 0.0, l21 = 0.0, l22 = 0.0;
    if (q_form == 1) {
        l11 = sqrt(q_c * dt * dt * dt / 3.0);
        l21 = (q_c * dt * dt / 2.0) / l11;
        l22 = sqrt(q_c * dt - l21 * l21);
    }
    for (int64_t b = 0; b < B; ++b) {
        const double* s = sensors + (sensors_per_traj ? 4 * b : 0);
        int64_t k0 = offsets[b], k1 = offsets[b + 1];
        double x[5];
        for (int i = 0; i < 5; ++i)
            x[i] = x0_mean[i] + x0_std[i] * normal01(seed, (uint64_t)b, 0, S_X0 + i);
        if (omega0_halfwidth > 0.0)
            x[4] = omega0_halfwidth * (2.0 * uniform01(seed, (uint64_t)b, 0, S_OMEGA0) - 1.0);
        for (int i = 0; i < 5; ++i) x_out[k0 * 5 + i] = x[i];
        y_out[k0 * 2 + 0] = 0.0;
        y_out[k0 * 2 + 1] = 0.0;
        for (int64_t k = k0 + 1; k < k1; ++k) {
            uint64_t step = (uint64_t)(k - k0);
            double nx[5];
            ct_propagate(x, dt, nx);
            double n[5];
            for (int i = 0; i < 5; ++i) n[i] = normal01(seed, (uint64_t)b, step, S_Q + i);
            if (q_form == 1) {
                nx[0] += l11 * n[0];
                nx[2] += l21 * n[0] + l22 * n[2];
                nx[1] += l11 * n[1];
                nx[3] += l21 * n[1] + l22 * n[3];
            } else {
                nx[2] += sqrt(q_c * dt) * n[2];
                nx[3] += sqrt(q_c * dt) * n[3];
            }
            nx[4] += sqrt(q_w * dt) * n[4];
            for (int i = 0; i < 5; ++i) x[i] = nx[i];
            for (int i = 0; i < 5; ++i) x_out[k * 5 + i] = x[i];
            for (int j = 0; j < 2; ++j) {
                double bear = atan2(x[1] - s[2 * j + 1], x[0] - s[2 * j]);
                y_out[k * 2 + j] = bear + r_std * normal01(seed, (uint64_t)b, step, S_R + j);
            }
        }
    }
}
