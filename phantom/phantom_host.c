/* Host build of the phantom generator: splits slices across threads. */
#include "phantom.h"
#include <pthread.h>
#include <stdlib.h>

typedef struct {
    const ph_desc* d;
    int16_t* out;
    int64_t z0, z1;
} ph_job;

static void* ph_worker(void* arg) {
    ph_job* j = (ph_job*)arg;
    const ph_desc* d = j->d;
    for (int64_t z = j->z0; z < j->z1; ++z)
        for (int64_t y = 0; y < d->ny; ++y) {
            int16_t* row = j->out + (z * d->ny + y) * d->nx;
            for (int64_t x = 0; x < d->nx; ++x) row[x] = ph_voxel(d, z, y, x);
        }
    return NULL;
}

int ph_generate_host(const ph_desc* d, int16_t* out, int nthreads) {
    if (!d || !out || d->nx <= 0 || d->ny <= 0 || d->nz <= 0) return 1;
    if (d->nx > 16384 || d->ny > 16384 || d->nz > 16384) return 1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > d->nz) nthreads = (int)d->nz;
    ph_job* jobs = (ph_job*)calloc((size_t)nthreads, sizeof(ph_job));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return 2; }
    for (int i = 0; i < nthreads; ++i) {
        jobs[i].d = d;
        jobs[i].out = out;
        jobs[i].z0 = d->nz * i / nthreads;
        jobs[i].z1 = d->nz * (i + 1) / nthreads;
    }
    int rc = 0;
    int started = 0;
    for (int i = 1; i < nthreads; ++i) {
        if (pthread_create(&th[i], NULL, ph_worker, &jobs[i]) != 0) { rc = 3; break; }
        started = i;
    }
    if (rc == 0) ph_worker(&jobs[0]);
    for (int i = 1; i <= started; ++i) pthread_join(th[i], NULL);
    free(jobs);
    free(th);
    return rc;
}
