/*
 * Fast, deterministic R-MAT edge generator for synthetic workloads (input
 * generation only: no part of the diffusion method is computed here).
 *
 * Sample i draws its quadrant at each of `scale` levels from a counter-based
 * stream: z = splitmix64(seed * 0x9E3779B97F4A7C15 + i * scale + level), and
 * r = ((z >> 32) * 100) >> 32 is uniform on {0..99} up to a bias below 1e-7.
 * Quadrant a when r < pa, b when r < pa + pb, c when r < pa + pb + pc, else d.
 * The result depends only on (scale, seed, i), not on the thread count or the
 * machine.  Keys are (src << 32) | dst; self-loops become UINT64_MAX.
 * sort_unique_u64 sorts keys (LSD radix, 16-bit digits) and drops duplicates
 * and UINT64_MAX, returning the number kept.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

typedef struct {
    int scale, pa, pb, pc;
    uint64_t seed;
    int64_t begin, end;
    uint64_t *keys;
} gen_job;

static void *gen_worker(void *arg)
{
    gen_job *j = (gen_job *)arg;
    const uint64_t base = j->seed * 0x9E3779B97F4A7C15ull;
    for (int64_t i = j->begin; i < j->end; ++i) {
        uint64_t src = 0, dst = 0;
        for (int l = 0; l < j->scale; ++l) {
            const uint64_t z = splitmix64(base + (uint64_t)i * (uint64_t)j->scale + (uint64_t)l);
            const uint32_t r = (uint32_t)(((z >> 32) * 100ull) >> 32);
            const uint64_t sbit = r >= (uint32_t)(j->pa + j->pb);
            const uint64_t dbit = (r >= (uint32_t)j->pa && r < (uint32_t)(j->pa + j->pb)) ||
                                  r >= (uint32_t)(j->pa + j->pb + j->pc);
            src = (src << 1) | sbit;
            dst = (dst << 1) | dbit;
        }
        j->keys[i] = src == dst ? UINT64_MAX : ((src << 32) | dst);
    }
    return NULL;
}

void rmat_keys(int scale, int64_t n_samples, int pa, int pb, int pc, uint64_t seed, int threads, uint64_t *keys)
{
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    pthread_t tid[256];
    gen_job jobs[256];
    for (int t = 0; t < threads; ++t) {
        jobs[t].scale = scale;
        jobs[t].pa = pa;
        jobs[t].pb = pb;
        jobs[t].pc = pc;
        jobs[t].seed = seed;
        jobs[t].begin = n_samples * t / threads;
        jobs[t].end = n_samples * (t + 1) / threads;
        jobs[t].keys = keys;
        pthread_create(&tid[t], NULL, gen_worker, &jobs[t]);
    }
    for (int t = 0; t < threads; ++t) pthread_join(tid[t], NULL);
}

/* ---------------------------------------------------------------- radix sort */
typedef struct {
    const uint64_t *in;
    uint64_t *out;
    int64_t begin, end;
    int shift;
    int64_t *hist; /* 65536 counts, then offsets */
} sort_job;

static void *hist_worker(void *arg)
{
    sort_job *j = (sort_job *)arg;
    memset(j->hist, 0, sizeof(int64_t) * 65536);
    for (int64_t i = j->begin; i < j->end; ++i) j->hist[(j->in[i] >> j->shift) & 0xFFFF]++;
    return NULL;
}

static void *scatter_worker(void *arg)
{
    sort_job *j = (sort_job *)arg;
    for (int64_t i = j->begin; i < j->end; ++i) {
        const uint64_t k = j->in[i];
        j->out[j->hist[(k >> j->shift) & 0xFFFF]++] = k;
    }
    return NULL;
}

int64_t sort_unique_u64(uint64_t *keys, uint64_t *tmp, int64_t n, int key_bits, int threads)
{
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    pthread_t tid[256];
    sort_job jobs[256];
    int64_t *hist = (int64_t *)malloc(sizeof(int64_t) * 65536 * (size_t)threads);
    if (!hist) return -1;
    uint64_t *a = keys, *b = tmp;
    /* UINT64_MAX marks dropped keys: it sorts last once all 64 bits are used, so
       sort all digits that can differ */
    const int passes = 4;
    (void)key_bits;
    for (int p = 0; p < passes; ++p) {
        for (int t = 0; t < threads; ++t) {
            jobs[t].in = a;
            jobs[t].out = b;
            jobs[t].begin = n * t / threads;
            jobs[t].end = n * (t + 1) / threads;
            jobs[t].shift = 16 * p;
            jobs[t].hist = hist + 65536 * (size_t)t;
            pthread_create(&tid[t], NULL, hist_worker, &jobs[t]);
        }
        for (int t = 0; t < threads; ++t) pthread_join(tid[t], NULL);
        int64_t off = 0;
        for (int d = 0; d < 65536; ++d)
            for (int t = 0; t < threads; ++t) {
                const int64_t c = hist[65536 * (size_t)t + d];
                hist[65536 * (size_t)t + d] = off;
                off += c;
            }
        for (int t = 0; t < threads; ++t) pthread_create(&tid[t], NULL, scatter_worker, &jobs[t]);
        for (int t = 0; t < threads; ++t) pthread_join(tid[t], NULL);
        uint64_t *x = a;
        a = b;
        b = x;
    }
    free(hist);
    /* after an even number of passes the sorted keys are back in `keys` */
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
        const uint64_t k = keys[i];
        if (k == UINT64_MAX) break;
        if (m == 0 || keys[m - 1] != k) keys[m++] = k;
    }
    return m;
}
