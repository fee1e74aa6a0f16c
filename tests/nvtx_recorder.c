/*
 * NVTX injection library used by the tests: it records every range push (its
 * message) and every range pop of the process it is injected into, one line
 * each, in the file named by NVTX_RECORD_FILE. NVTX 3 loads it when
 * NVTX_INJECTION64_PATH names it and calls InitializeInjectionNvtx2, which
 * replaces the core module's RangePushA and RangePop entries through the
 * callback export table. Built by tests/test_abi.py with gcc.
 */
#include <stdio.h>
#include <stdlib.h>

#include <nvtx3/nvToolsExt.h>

static FILE *g_out;

static int record_push(const char *message)
{
    if (g_out) {
        fprintf(g_out, "push %s\n", message ? message : "");
        fflush(g_out);
    }
    return 0;
}

static int record_pop(void)
{
    if (g_out) {
        fputs("pop\n", g_out);
        fflush(g_out);
    }
    return 0;
}

__attribute__((visibility("default"))) int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_table)
{
    const NvtxExportTableCallbacks *cb = (const NvtxExportTableCallbacks *)get_table(NVTX_ETID_CALLBACKS);
    NvtxFunctionTable table = 0;
    unsigned int last = 0;
    if (!cb || !cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE, &table, &last) || !table)
        return 0;
    if (last < NVTX_CBID_CORE_RangePushA || last < NVTX_CBID_CORE_RangePop)
        return 0;
    const char *path = getenv("NVTX_RECORD_FILE");
    g_out = path ? fopen(path, "w") : NULL;
    *table[NVTX_CBID_CORE_RangePushA] = (NvtxFunctionPointer)record_push;
    *table[NVTX_CBID_CORE_RangePop] = (NvtxFunctionPointer)record_pop;
    return 1;
}
