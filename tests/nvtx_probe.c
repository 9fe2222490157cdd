/* Test helper: an NVTX injection library (loaded through
 * NVTX_INJECTION64_PATH) that records every range push and pop of the
 * process, so that a CPU test can see which NVTX ranges libpgm opens
 * without Nsight Systems.  Registers its handlers in the CORE callback
 * table that the NVTX headers export to injections. */
#include <nvtx3/nvToolsExt.h>
#include <string.h>

static char g_log[1 << 16];
static size_t g_len = 0;
static int g_depth = 0, g_max_depth = 0, g_pops = 0;

static int probe_push(const char *msg) {
  size_t n = msg ? strlen(msg) : 0;
  if (g_len + n + 2 < sizeof(g_log)) {
    memcpy(g_log + g_len, msg, n);
    g_len += n;
    g_log[g_len++] = '\n';
    g_log[g_len] = 0;
  }
  if (++g_depth > g_max_depth) g_max_depth = g_depth;
  return g_depth - 1;
}

static int probe_pop(void) {
  g_pops++;
  return --g_depth;
}

int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get) {
  const NvtxExportTableCallbacks *cb = (const NvtxExportTableCallbacks *)get(NVTX_ETID_CALLBACKS);
  NvtxFunctionTable table = 0;
  unsigned int size = 0;
  if (!cb || !cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE, &table, &size) || !table) return 0;
  if (size <= NVTX_CBID_CORE_RangePop) return 0;
  *table[NVTX_CBID_CORE_RangePushA] = (NvtxFunctionPointer)probe_push;
  *table[NVTX_CBID_CORE_RangePop] = (NvtxFunctionPointer)probe_pop;
  return 1;
}

/* the recorded range names (one per line), the current and largest depth, and the pops */
const char *nvtx_probe_log(void) { return g_log; }
int nvtx_probe_depth(void) { return g_depth; }
int nvtx_probe_max_depth(void) { return g_max_depth; }
int nvtx_probe_pops(void) { return g_pops; }
