"""FP64 CPU oracle for the LSNIF query (test infrastructure only)."""
