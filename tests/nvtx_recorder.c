/*
 * NVTX injection library used by tests/test_gpu_nvtx.py (test
 * infrastructure, not part of the library).  NVTX v3 loads the shared
 * library named by NVTX_INJECTION64_PATH the first time a module calls an
 * NVTX function and calls its InitializeInjectionNvtx2; this one replaces
 * the core module's RangePushA and RangePop with functions that append
 * "push <name>" and "pop" lines to the file named by PDOT_NVTX_LOG.
 */
#define NVTX_NO_IMPL
#include <nvtx3/nvToolsExt.h>

#include <pthread.h>
#include <stdio.h>
#include <stdlib.h>

static FILE *g_log;
static pthread_mutex_t g_lock = PTHREAD_MUTEX_INITIALIZER;

static int rec_push(const char *name) {
    pthread_mutex_lock(&g_lock);
    if (g_log) {
        fprintf(g_log, "push %s\n", name ? name : "");
        fflush(g_log);
    }
    pthread_mutex_unlock(&g_lock);
    return 0;
}

static int rec_pop(void) {
    pthread_mutex_lock(&g_lock);
    if (g_log) {
        fputs("pop\n", g_log);
        fflush(g_log);
    }
    pthread_mutex_unlock(&g_lock);
    return 0;
}

__attribute__((visibility("default"))) int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_table) {
    const char *path = getenv("PDOT_NVTX_LOG");
    if (!path || !get_table) return 0;
    pthread_mutex_lock(&g_lock);
    if (!g_log) g_log = fopen(path, "a");
    const int ok = g_log != NULL;
    pthread_mutex_unlock(&g_lock);
    if (!ok) return 0;
    const NvtxExportTableCallbacks *cb = (const NvtxExportTableCallbacks *)get_table(NVTX_ETID_CALLBACKS);
    NvtxFunctionTable table = NULL;
    unsigned int size = 0;
    if (!cb || !cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE, &table, &size) || !table) return 0;
    if (size < NVTX_CBID_CORE_RangePop) return 0;
    *table[NVTX_CBID_CORE_RangePushA] = (NvtxFunctionPointer)rec_push;
    *table[NVTX_CBID_CORE_RangePop] = (NvtxFunctionPointer)rec_pop;
    return 1;
}
