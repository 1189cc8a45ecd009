/* abi_c_client.c -- a plain C99 caller of libqtask.so through include/qtask.h
 * alone: no Python, no PyTorch, no C++.  It builds the GHZ circuit (H on q0,
 * then a CNOT chain, one level per gate), checks the ABI's host-side
 * contract (conflict detection leaves the circuit unchanged, level counts,
 * argument errors with messages, stale reads after a dry run) and plans one
 * update in dry-run mode, which launches nothing and needs no GPU.
 * Exit status 0 and "ok" on success; a distinct non-zero code per failed
 * check otherwise. */
#include <stdio.h>
#include <string.h>

#include "qtask.h"

static qt_gate one_target(int32_t kind, int32_t t) {
    qt_gate g;
    memset(&g, 0, sizeof g);
    g.kind = kind;
    g.ntarget = 1;
    g.target[0] = t;
    return g;
}

int main(void) {
    const int32_t n = 10;
    qt_circuit* c = NULL;
    if (qt_create(n, QT_C128_DF, 4, &c) != QT_OK || !c) return 1;
    if (qt_set_option(c, "dry_run", 1) != QT_OK) return 2;

    qt_gate_id id = 0, first = 0;
    qt_gate h = one_target(QT_H, 0);
    if (qt_insert_level(c, 0) != QT_OK) return 3;
    if (qt_insert_gate(c, 0, &h, &first) != QT_OK) return 4;
    for (int32_t q = 0; q + 1 < n; ++q) {
        qt_gate cx = one_target(QT_CNOT, q + 1);
        cx.ncontrol = 1;
        cx.control[0] = q;
        if (qt_insert_level(c, q + 1) != QT_OK) return 5;
        if (qt_insert_gate(c, q + 1, &cx, &id) != QT_OK) return 6;
    }
    int32_t levels = 0;
    int64_t gates = 0;
    if (qt_num_levels(c, &levels) != QT_OK || levels != n) return 7;
    if (qt_num_gates(c, &gates) != QT_OK || gates != n) return 8;

    /* a gate sharing q0 with the H of level 0: rejected, circuit unchanged */
    qt_gate x = one_target(QT_X, 0);
    if (qt_insert_gate(c, 0, &x, &id) != QT_ERR_CONFLICT) return 9;
    if (qt_num_gates(c, &gates) != QT_OK || gates != n) return 10;
    const char* msg = qt_last_error(c);
    if (!msg || !msg[0]) return 11;

    /* argument errors: qubit out of range, unknown option */
    qt_gate bad = one_target(QT_X, n);
    if (qt_insert_gate(c, 1, &bad, &id) != QT_ERR_ARG) return 12;
    if (qt_set_option(c, "no_such_option", 1) == QT_OK) return 13;

    /* plan the update (dry run: launches are planned and counted, none is
     * issued, nothing is allocated) */
    qt_update_stats st;
    memset(&st, 0, sizeof st);
    if (qt_update_state(c, 0, &st) != QT_OK) return 14;
    if (st.gates_total != n || st.passes_total < 1) return 15;
    if (st.amp_updates != (uint64_t)n << n) return 16;

    /* the dry run computed no state: reading it is stale */
    double amp[2];
    if (qt_read_amplitudes(c, 0, 1, amp) != QT_ERR_STALE) return 17;

    /* remove the H again: the edit is accepted and the next plan counts one gate fewer */
    if (qt_remove_gate(c, 0, first) != QT_OK) return 18;
    if (qt_update_state(c, 0, &st) != QT_OK || st.gates_total != n - 1) return 19;

    if (qt_destroy(c) != QT_OK) return 20;
    /* creation errors carry a message under the NULL handle */
    qt_circuit* none = NULL;
    if (qt_create(0, QT_C64, 0, &none) != QT_ERR_ARG || none) return 21;
    msg = qt_last_error(NULL);
    if (!msg || !strstr(msg, "n_qubits")) return 22;
    printf("ok\n");
    return 0;
}
