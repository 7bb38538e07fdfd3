/* Host (C, OpenMP) R-MAT generator: the same recipe as graphgen.rmat, value for value.
 *
 * Edge e (0 <= e < M) descends `scale` quadrant levels; level l draws u = hash(seed, e*scale+l)
 * (the counter-based hash below) and compares it with the 32-bit thresholds ta <= tab <= tabc:
 * the source bit is u >= tab, the destination bit is (ta <= u < tab) or u >= tabc (thresholds
 * up to 2^32, so compared in 64 bits).  Vertex IDs
 * are then relabelled through the permutation that sorts the keys (hash(pseed, v) << 31) | v
 * (when pseed >= 0), self loops and duplicate edges are dropped and the CSR is sorted by
 * (source, destination).  Input generation only: nothing of the graph algorithms is here.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint32_t lowbias32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7FEB352Du;
    x ^= x >> 15;
    x *= 0x846CA68Bu;
    x ^= x >> 16;
    return x;
}

static inline uint32_t hash_u32(uint32_t s, uint32_t k, uint64_t counter) {
    const uint32_t lo = (uint32_t)(counter & 0xFFFFFFFFu), hi = (uint32_t)(counter >> 32);
    uint32_t h = lowbias32(lo ^ k);
    return lowbias32(h ^ (uint32_t)(hi + 0x68E31DA4u + s));
}

static inline uint32_t seed_key(uint32_t s) { return lowbias32(s ^ 0x9E3779B9u); }

/* LSD radix sort of 64-bit keys by their low `bits` bits (8 bits per pass), into `a` */
static void radix_sort_u64(uint64_t *a, uint64_t *tmp, int64_t n, int bits) {
    for (int shift = 0; shift < bits; shift += 8) {
        int64_t cnt[257];
        memset(cnt, 0, sizeof cnt);
        for (int64_t i = 0; i < n; ++i) ++cnt[((a[i] >> shift) & 0xFF) + 1];
        for (int b = 0; b < 256; ++b) cnt[b + 1] += cnt[b];
        for (int64_t i = 0; i < n; ++i) tmp[cnt[(a[i] >> shift) & 0xFF]++] = a[i];
        memcpy(a, tmp, (size_t)n * 8);
    }
}

static int cmp_i32(const void *x, const void *y) {
    const int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
    return (a > b) - (a < b);
}

/* rowptr: int64[V + 1] out; *colidx_out: int32[E] allocated here (free with gg_free).
 * Returns E, or -1 when memory runs out. */
int64_t gg_rmat(int scale, int64_t edge_factor, uint64_t ta, uint64_t tab, uint64_t tabc, int64_t seed,
                int64_t pseed, int64_t *rowptr, int32_t **colidx_out) {
    const int64_t V = (int64_t)1 << scale, M = edge_factor * V;
    const uint32_t s = (uint32_t)seed, k = seed_key(s);
    int32_t *src = (int32_t *)malloc((size_t)M * 4), *dst = (int32_t *)malloc((size_t)M * 4);
    int32_t *perm = (int32_t *)malloc((size_t)V * 4);
    if (!src || !dst || !perm) {
        free(src), free(dst), free(perm);
        return -1;
    }
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < M; ++e) {
        uint32_t sv = 0, dv = 0;
        for (int l = 0; l < scale; ++l) {
            const uint64_t u = hash_u32(s, k, (uint64_t)e * (uint64_t)scale + (uint64_t)l);
            sv = (sv << 1) | (uint32_t)(u >= tab);
            dv = (dv << 1) | (uint32_t)((u >= ta && u < tab) || u >= tabc);
        }
        src[e] = (int32_t)sv;
        dst[e] = (int32_t)dv;
    }
    if (pseed >= 0) {  /* perm[i] = the vertex with the i-th smallest key */
        uint64_t *key = (uint64_t *)malloc((size_t)V * 8), *tmp = (uint64_t *)malloc((size_t)V * 8);
        if (!key || !tmp) {
            free(key), free(tmp), free(src), free(dst), free(perm);
            return -1;
        }
        const uint32_t ps = (uint32_t)pseed, pk = seed_key(ps);
#pragma omp parallel for schedule(static)
        for (int64_t v = 0; v < V; ++v) key[v] = ((uint64_t)hash_u32(ps, pk, (uint64_t)v) << 31) | (uint64_t)v;
        radix_sort_u64(key, tmp, V, 64);
        for (int64_t i = 0; i < V; ++i) perm[i] = (int32_t)(key[i] & 0x7FFFFFFFu);
        free(key), free(tmp);
#pragma omp parallel for schedule(static)
        for (int64_t e = 0; e < M; ++e) {
            src[e] = perm[src[e]];
            dst[e] = perm[dst[e]];
        }
    }
    free(perm);
    /* bucket by source, then sort and deduplicate every row */
    int64_t *cnt = (int64_t *)calloc((size_t)V + 1, 8);
    int32_t *col = (int32_t *)malloc((size_t)M * 4);
    if (!cnt || !col) {
        free(cnt), free(col), free(src), free(dst);
        return -1;
    }
    for (int64_t e = 0; e < M; ++e)
        if (src[e] != dst[e]) ++cnt[src[e] + 1];
    for (int64_t v = 0; v < V; ++v) cnt[v + 1] += cnt[v];
    int64_t *pos = (int64_t *)malloc((size_t)V * 8);
    if (!pos) {
        free(cnt), free(col), free(src), free(dst);
        return -1;
    }
    memcpy(pos, cnt, (size_t)V * 8);
    for (int64_t e = 0; e < M; ++e)
        if (src[e] != dst[e]) col[pos[src[e]]++] = dst[e];
    free(src), free(dst), free(pos);
    int64_t *len = (int64_t *)malloc((size_t)V * 8);
    if (!len) {
        free(cnt), free(col);
        return -1;
    }
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t v = 0; v < V; ++v) {
        int32_t *r = col + cnt[v];
        const int64_t n = cnt[v + 1] - cnt[v];
        qsort(r, (size_t)n, 4, cmp_i32);
        int64_t m = 0;
        for (int64_t i = 0; i < n; ++i)
            if (m == 0 || r[i] != r[m - 1]) r[m++] = r[i];
        len[v] = m;
    }
    rowptr[0] = 0;
    for (int64_t v = 0; v < V; ++v) rowptr[v + 1] = rowptr[v] + len[v];
    const int64_t E = rowptr[V];
    int32_t *out = (int32_t *)malloc((size_t)(E > 0 ? E : 1) * 4);
    if (!out) {
        free(cnt), free(col), free(len);
        return -1;
    }
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t v = 0; v < V; ++v) memcpy(out + rowptr[v], col + cnt[v], (size_t)len[v] * 4);
    free(cnt), free(col), free(len);
    *colidx_out = out;
    return E;
}

void gg_free(void *p) { free(p); }
