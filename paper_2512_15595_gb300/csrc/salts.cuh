// Generated by gen_salts.py -- do not edit.
// Odd multipliers for the salted multiplicative bit positions (Sec. IV-B).
// salt64[i] = SplitMix64(seed 0x5A175EED) output i, low bit set;
// salt32[i] = (salt64[i] >> 32) | 1.
#pragma once
#include <cstdint>
namespace bloomgb {
constexpr int kMaxSalts = 64;
__host__ __device__ constexpr uint64_t salt64_at(int i) {
  switch (i) {
    case 0: return 0x543FE2D36F7B9D77ull;
    case 1: return 0x034B77665B2ECBB5ull;
    case 2: return 0x5BE4C04A31F09855ull;
    case 3: return 0xBE05210299D26B3Bull;
    case 4: return 0xEE3ACC25A0D0A021ull;
    case 5: return 0xAE4A043CF60FE9C3ull;
    case 6: return 0x78786A09806CDFA1ull;
    case 7: return 0x5E474993DD5A58FBull;
    case 8: return 0xCACBA5A05B81F27Full;
    case 9: return 0x25BC41996E6C65DBull;
    case 10: return 0xE0B4AA719F60B935ull;
    case 11: return 0xE4B87130A366CCFBull;
    case 12: return 0x4247BF906211533Dull;
    case 13: return 0xB9299BAD7DB0182Dull;
    case 14: return 0xCD5F70E99AB32BB7ull;
    case 15: return 0x3EF6B382029D326Full;
    case 16: return 0x6981C98E3D72EB99ull;
    case 17: return 0xDDBDD1BD480A2BB7ull;
    case 18: return 0x68FABFE33699E91Bull;
    case 19: return 0xFA71F68EAEF65413ull;
    case 20: return 0xC47220AA9CED1DA9ull;
    case 21: return 0x618CB4CA21296C53ull;
    case 22: return 0xBC9A4784480F56F7ull;
    case 23: return 0x637ADB3B5F0E49D9ull;
    case 24: return 0x0EC5B8F150F77149ull;
    case 25: return 0xBC9905E7E77A8BBFull;
    case 26: return 0x29985BE7ECA9041Dull;
    case 27: return 0x1C5AF343D10C1565ull;
    case 28: return 0xE38C9D4C88A197A9ull;
    case 29: return 0x6839117133C47885ull;
    case 30: return 0x169E76C3645A44E1ull;
    case 31: return 0x0BFF5816EB57C36Full;
    case 32: return 0x2D95CB8869EB0E35ull;
    case 33: return 0x1DAD55053B121D71ull;
    case 34: return 0x2729F3937F63EB3Full;
    case 35: return 0x467F9EC381AAA2B9ull;
    case 36: return 0x28F0E05168C0A873ull;
    case 37: return 0xFD03AF6B0174380Full;
    case 38: return 0xEA8D89CE71EA27B9ull;
    case 39: return 0x43E3D61547DE97F5ull;
    case 40: return 0x658C108F93B2B9D1ull;
    case 41: return 0x62E92B5F6FA92001ull;
    case 42: return 0x3B8C82D87DB87827ull;
    case 43: return 0xDC219001C4BCE2DBull;
    case 44: return 0xF214993652D748EBull;
    case 45: return 0xC54C0187C39332DDull;
    case 46: return 0xD626DB5F1280B551ull;
    case 47: return 0x8982938CF8ED53C9ull;
    case 48: return 0x2F2DE8BBD0969203ull;
    case 49: return 0x36216A37817ADF23ull;
    case 50: return 0x0D14A2AB29F4812Full;
    case 51: return 0x44B3424AA5016207ull;
    case 52: return 0x78A71A3433C6B28Bull;
    case 53: return 0x2192A132AE152FBBull;
    case 54: return 0x63FE9418246CDCA9ull;
    case 55: return 0x8D40CA93119D98F9ull;
    case 56: return 0x00FCFFD8672489B5ull;
    case 57: return 0xD0C99D2ED33BAE7Bull;
    case 58: return 0xBD031D6AB1CAB1B5ull;
    case 59: return 0xC70087A386612BE1ull;
    case 60: return 0x50C742314088A783ull;
    case 61: return 0xA57297428EA07B09ull;
    case 62: return 0x90E42F851A57004Bull;
    case 63: return 0xBB9BCB437A21D2C7ull;
    default: return 0;
  }
}
__host__ __device__ constexpr uint32_t salt32_at(int i) {
  switch (i) {
    case 0: return 0x543FE2D3u;
    case 1: return 0x034B7767u;
    case 2: return 0x5BE4C04Bu;
    case 3: return 0xBE052103u;
    case 4: return 0xEE3ACC25u;
    case 5: return 0xAE4A043Du;
    case 6: return 0x78786A09u;
    case 7: return 0x5E474993u;
    case 8: return 0xCACBA5A1u;
    case 9: return 0x25BC4199u;
    case 10: return 0xE0B4AA71u;
    case 11: return 0xE4B87131u;
    case 12: return 0x4247BF91u;
    case 13: return 0xB9299BADu;
    case 14: return 0xCD5F70E9u;
    case 15: return 0x3EF6B383u;
    case 16: return 0x6981C98Fu;
    case 17: return 0xDDBDD1BDu;
    case 18: return 0x68FABFE3u;
    case 19: return 0xFA71F68Fu;
    case 20: return 0xC47220ABu;
    case 21: return 0x618CB4CBu;
    case 22: return 0xBC9A4785u;
    case 23: return 0x637ADB3Bu;
    case 24: return 0x0EC5B8F1u;
    case 25: return 0xBC9905E7u;
    case 26: return 0x29985BE7u;
    case 27: return 0x1C5AF343u;
    case 28: return 0xE38C9D4Du;
    case 29: return 0x68391171u;
    case 30: return 0x169E76C3u;
    case 31: return 0x0BFF5817u;
    case 32: return 0x2D95CB89u;
    case 33: return 0x1DAD5505u;
    case 34: return 0x2729F393u;
    case 35: return 0x467F9EC3u;
    case 36: return 0x28F0E051u;
    case 37: return 0xFD03AF6Bu;
    case 38: return 0xEA8D89CFu;
    case 39: return 0x43E3D615u;
    case 40: return 0x658C108Fu;
    case 41: return 0x62E92B5Fu;
    case 42: return 0x3B8C82D9u;
    case 43: return 0xDC219001u;
    case 44: return 0xF2149937u;
    case 45: return 0xC54C0187u;
    case 46: return 0xD626DB5Fu;
    case 47: return 0x8982938Du;
    case 48: return 0x2F2DE8BBu;
    case 49: return 0x36216A37u;
    case 50: return 0x0D14A2ABu;
    case 51: return 0x44B3424Bu;
    case 52: return 0x78A71A35u;
    case 53: return 0x2192A133u;
    case 54: return 0x63FE9419u;
    case 55: return 0x8D40CA93u;
    case 56: return 0x00FCFFD9u;
    case 57: return 0xD0C99D2Fu;
    case 58: return 0xBD031D6Bu;
    case 59: return 0xC70087A3u;
    case 60: return 0x50C74231u;
    case 61: return 0xA5729743u;
    case 62: return 0x90E42F85u;
    case 63: return 0xBB9BCB43u;
    default: return 0;
  }
}
}  // namespace bloomgb
