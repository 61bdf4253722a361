/* nvtx_probe.c -- a minimal NVTX tool for the tests (not part of the library).
 *
 * Loaded by NVTX itself when the environment names it in
 * NVTX_INJECTION64_PATH: the NVTX headers that a program is built with look
 * that variable up on the first NVTX call and call the tool's
 * InitializeInjectionNvtx2, which installs its own handlers for the core
 * calls (push / pop, marks, start / end of process-wide ranges).  This probe
 * counts every message it sees and, at exit, writes one line per
 * "kind message" with its count to the file named by PTG_NVTX_LOG.
 *
 * Build: gcc -shared -fPIC -O2 -I<cuda>/include nvtx_probe.c -o nvtx_probe.so -lpthread
 */
#include <nvtx3/nvToolsExt.h>
#include <pthread.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define PROBE_MAX 256

static struct {
    char key[96];
    long count;
} g_seen[PROBE_MAX];
static int g_nseen = 0;
static pthread_mutex_t g_mu = PTHREAD_MUTEX_INITIALIZER;
static unsigned long long g_next_range = 1;
static int g_atexit_done = 0;

static void bump(const char* kind, const char* msg)
{
    char key[96];
    snprintf(key, sizeof key, "%s %s", kind, msg ? msg : "");
    pthread_mutex_lock(&g_mu);
    int k = 0;
    while (k < g_nseen && strcmp(g_seen[k].key, key) != 0) ++k;
    if (k == g_nseen && g_nseen < PROBE_MAX) {
        strcpy(g_seen[k].key, key);
        g_seen[k].count = 0;
        ++g_nseen;
    }
    if (k < g_nseen) ++g_seen[k].count;
    pthread_mutex_unlock(&g_mu);
}

static int probe_push_a(const char* msg)
{
    bump("push", msg);
    return 0;
}

static int probe_pop(void)
{
    bump("pop", "");
    return 0;
}

static void probe_mark_a(const char* msg) { bump("mark", msg); }

static nvtxRangeId_t probe_start_a(const char* msg)
{
    bump("start", msg);
    pthread_mutex_lock(&g_mu);
    const nvtxRangeId_t id = g_next_range++;
    pthread_mutex_unlock(&g_mu);
    return id;
}

static void probe_end(nvtxRangeId_t id)
{
    (void)id;
    bump("end", "");
}

static void dump(void)
{
    const char* path = getenv("PTG_NVTX_LOG");
    if (!path) return;
    FILE* f = fopen(path, "w");
    if (!f) return;
    pthread_mutex_lock(&g_mu);
    for (int k = 0; k < g_nseen; ++k) fprintf(f, "%s\t%ld\n", g_seen[k].key, g_seen[k].count);
    pthread_mutex_unlock(&g_mu);
    fclose(f);
}

int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_table)
{
    const NvtxExportTableCallbacks* cb = (const NvtxExportTableCallbacks*)get_table(NVTX_ETID_CALLBACKS);
    NvtxFunctionTable table = NULL;
    unsigned int last = 0;
    if (!cb || !cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE, &table, &last) || !table) return 0;
    if (last < NVTX_CBID_CORE_RangePop) return 0;
    *table[NVTX_CBID_CORE_MarkA] = (NvtxFunctionPointer)probe_mark_a;
    *table[NVTX_CBID_CORE_RangeStartA] = (NvtxFunctionPointer)probe_start_a;
    *table[NVTX_CBID_CORE_RangeEnd] = (NvtxFunctionPointer)probe_end;
    *table[NVTX_CBID_CORE_RangePushA] = (NvtxFunctionPointer)probe_push_a;
    *table[NVTX_CBID_CORE_RangePop] = (NvtxFunctionPointer)probe_pop;
    pthread_mutex_lock(&g_mu);
    const int first = !g_atexit_done;
    g_atexit_done = 1;
    pthread_mutex_unlock(&g_mu);
    if (first) atexit(dump);
    return 1;
}
