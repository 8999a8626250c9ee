"""ORACLE - TEST INFRASTRUCTURE ONLY: the plain FP64 CPU restatement of the
method.  Importable only by tests, the smoke check and the benchmark's CPU
baseline."""
