"""CPU oracle for batch-dynamic subgraph matching (test infrastructure only;
never imported by the library)."""
