"""CPU oracle for exact reverse k-MIPS (test infrastructure; never on the product path)."""
