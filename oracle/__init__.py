"""Serial FP64 CPU oracle for Vertex Block Descent (test infrastructure only)."""
