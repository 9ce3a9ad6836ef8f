/*
 * Exact triangle count of a simple undirected graph (oracle helper).
 *
 * TEST INFRASTRUCTURE ONLY: used to report the relative error of the
 * estimate against tau(G) (Sec. 2 defines tau as the number of triangles).
 * Nothing in the product path links this file.
 *
 * Method: the "forward" algorithm -- orient every edge from the endpoint of
 * lower (degree, id) to the higher one, so every triangle is counted exactly
 * once at its lowest vertex as a common out-neighbour of two oriented edges;
 * out-lists are sorted and intersected by merging.  Work O(m^{3/2}).
 *
 * Pins: brute-force enumeration and trace(A^3)/6 on random graphs, closed
 * forms for complete, bipartite and wheel graphs (tests/test_oracle_exact.py).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int cmp_u32(const void *a, const void *b) {
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return (x > y) - (x < y);
}

/* keys: m packed edges (u << 32) | v with u < v < n.  Returns tau, or
 * UINT64_MAX when memory runs out. */
uint64_t oracle_count_triangles(const uint64_t *keys, uint64_t m, uint32_t n) {
    uint64_t *deg = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    uint64_t *off = (uint64_t *)calloc((size_t)n + 2, sizeof(uint64_t));
    uint32_t *adj = (uint32_t *)malloc((m ? m : 1) * sizeof(uint32_t));
    uint64_t *fill = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    if (!deg || !off || !adj || !fill) {
        free(deg); free(off); free(adj); free(fill);
        return UINT64_MAX;
    }
    for (uint64_t i = 0; i < m; ++i) {
        deg[keys[i] >> 32]++;
        deg[keys[i] & 0xffffffffu]++;
    }
    /* a precedes b when (deg a, a) < (deg b, b) */
#define BEFORE(a, b) (deg[a] < deg[b] || (deg[a] == deg[b] && (a) < (b)))
    for (uint64_t i = 0; i < m; ++i) {
        uint32_t a = (uint32_t)(keys[i] >> 32), b = (uint32_t)(keys[i] & 0xffffffffu);
        uint32_t lo = BEFORE(a, b) ? a : b;
        off[lo + 1]++;
    }
    for (uint32_t x = 0; x < n; ++x) off[x + 1] += off[x];
    for (uint64_t i = 0; i < m; ++i) {
        uint32_t a = (uint32_t)(keys[i] >> 32), b = (uint32_t)(keys[i] & 0xffffffffu);
        uint32_t lo = BEFORE(a, b) ? a : b, hi = (lo == a) ? b : a;
        adj[off[lo] + fill[lo]++] = hi;
    }
#undef BEFORE
    for (uint32_t x = 0; x < n; ++x)
        qsort(adj + off[x], (size_t)(off[x + 1] - off[x]), sizeof(uint32_t), cmp_u32);
    uint64_t tau = 0;
    for (uint32_t a = 0; a < n; ++a) {
        for (uint64_t k = off[a]; k < off[a + 1]; ++k) {
            uint32_t b = adj[k];
            uint64_t i = off[a], iend = off[a + 1];
            uint64_t j = off[b], jend = off[b + 1];
            while (i < iend && j < jend) {
                if (adj[i] < adj[j]) ++i;
                else if (adj[i] > adj[j]) ++j;
                else { ++tau; ++i; ++j; }
            }
        }
    }
    free(deg); free(off); free(adj); free(fill);
    return tau;
}
