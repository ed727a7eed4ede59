"""CPU oracle for the weighted-ensemble Gillespie-SSA path (arXiv:1303.5986).

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the benchmark's CPU
baseline leg use it; the product library never does.  ``oracle.oracle`` wraps the plain C
implementation (``we_oracle.c``); ``oracle.exact`` holds closed forms and master-equation
solutions that pin the oracle to the mathematics.
"""
