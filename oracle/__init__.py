"""CPU FP64 oracle for SP2 purification -- test infrastructure only.

Only the tests, the smoke check and the benchmark's CPU-baseline leg import this
package; the library never does.
"""
