/* Exact enumeration of the periodic Ising torus (test infrastructure only).
 *
 * Z = sum over all 2^(Lx*Ly) spin configurations of
 *     exp(beta J sum_<ij> s_i s_j + beta h sum_i s_i)        (SM Sec. A)
 * with bonds i -> i + x (mod Lx) and i -> i + y (mod Ly) for every site, so a
 * side of length 2 carries doubled bonds, exactly like a 2-wide tensor
 * network torus.  Instead of summing exponentials this returns the integer
 * density of states g[b][m]: the number of configurations with bond sum
 * b - 2n and magnetisation m - n (n = Lx*Ly), which callers turn into
 * ln Z and its derivatives in floating point.  g must hold
 * (4n + 1) * (2n + 1) int64 entries.  Returns 0, or -1 for n outside 1..30.
 */
#include <stdint.h>
#include <string.h>

int ising_density_of_states(int Lx, int Ly, int64_t *g)
{
    const int n = Lx * Ly;
    if (Lx < 1 || Ly < 1 || n > 30) return -1;
    const int nm = 2 * n + 1;
    memset(g, 0, sizeof(int64_t) * (size_t)(4 * n + 1) * (size_t)nm);
    const uint64_t states = (uint64_t)1 << n;
    for (uint64_t c = 0; c < states; ++c) {
        int bonds = 0, mag = 0;
        for (int y = 0; y < Ly; ++y) {
            for (int x = 0; x < Lx; ++x) {
                const int i = y * Lx + x;
                const int si = ((c >> i) & 1u) ? -1 : 1;
                const int jx = y * Lx + (x + 1) % Lx;
                const int jy = ((y + 1) % Ly) * Lx + x;
                const int sx = ((c >> jx) & 1u) ? -1 : 1;
                const int sy = ((c >> jy) & 1u) ? -1 : 1;
                bonds += si * sx + si * sy;
                mag += si;
            }
        }
        g[(size_t)(bonds + 2 * n) * nm + (size_t)(mag + n)] += 1;
    }
    return 0;
}
