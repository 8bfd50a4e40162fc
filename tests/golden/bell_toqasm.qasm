// QCLAB Sec. 4: the toQASM output the paper prints for its example circuit of Sec. 2
// (H on q0, CNOT q0 -> q1, measure q0, measure q1).
qreg q[2];
h q[0];
cx q[0], q[1];
measure q[0];
measure q[1];
