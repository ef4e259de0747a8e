/*
 * Hard-disk Metropolis in a periodic square box (Metropolis et al. 1953):
 * test helper giving an independent pressure estimate for the ECMC oracle.
 * Moves: one disk, uniform displacement in [-delta, delta]^2, rejected on
 * overlap. Measurement: histogram of pair distances r in [d, d + nb*dr);
 * the contact value g(d+) of the pair correlation gives the 2D virial
 * pressure beta P / rho = 1 + (pi/2) rho d^2 g(d+).
 * Random numbers: SplitMix64 (counter form) mapped to doubles in [0, 1).
 */
#include <math.h>
#include <stdint.h>

static uint64_t sm_state;

static double urand(void) {
    uint64_t z = (sm_state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * 0x1.0p-53;
}

static double pdist2(double ax, double ay, double bx, double by, double L) {
    double dx = fabs(ax - bx), dy = fabs(ay - by);
    if (dx > L - dx) dx = L - dx;
    if (dy > L - dy) dy = L - dy;
    return dx * dx + dy * dy;
}

/* Runs `sweeps` sweeps (n moves each) after `burn` sweeps, measuring the
   histogram every `every` sweeps. hist[nb] counts pairs with r in bins of dr.
   Returns the acceptance rate. x, y are updated in place. */
double metro_run(int n, double L, double d, double *x, double *y, double delta,
                 long burn, long sweeps, int every, int nb, double dr, double *hist,
                 uint64_t seed) {
    sm_state = seed;
    long acc = 0, tries = 0;
    const double d2 = d * d;
    for (long s = 0; s < burn + sweeps; ++s) {
        for (int m = 0; m < n; ++m) {
            int i = (int)(urand() * n);
            double nx = x[i] + (2.0 * urand() - 1.0) * delta;
            double ny = y[i] + (2.0 * urand() - 1.0) * delta;
            nx -= L * floor(nx / L);
            ny -= L * floor(ny / L);
            int ok = 1;
            for (int j = 0; j < n && ok; ++j)
                if (j != i && pdist2(nx, ny, x[j], y[j], L) < d2) ok = 0;
            ++tries;
            if (ok) {
                x[i] = nx;
                y[i] = ny;
                ++acc;
            }
        }
        if (s >= burn && (s - burn) % every == 0) {
            for (int i = 0; i < n; ++i)
                for (int j = i + 1; j < n; ++j) {
                    double r = sqrt(pdist2(x[i], y[i], x[j], y[j], L));
                    int b = (int)((r - d) / dr);
                    if (r >= d && b < nb) hist[b] += 1.0;
                }
        }
    }
    return (double)acc / (double)tries;
}
